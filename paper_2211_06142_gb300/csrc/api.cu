// api.cu -- host side of the C ABI declared in include/cgdem.h: parameter
// derivation (coarse-graining rules, Sec. 2.4), workspace layout, the verbs
// of the step and their CUDA-graph schedule.
#include <algorithm>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "cgdem_internal.cuh"

namespace cgdem {
void launch_forces(const Dev& d, int mode, int block, cudaStream_t s, cudaGraphConditionalHandle h_next,
                   cudaGraphConditionalHandle h_fluid = 0);
void launch_rebuild(const Dev& d, cudaStream_t s);
void launch_set_rebuild(const Dev& d, cudaStream_t s);
void launch_rebuild_cond(const Dev& d, cudaGraphConditionalHandle h, cudaStream_t s);
void launch_bond_touching(const Dev& d, cudaStream_t s);
void launch_couple(const Dev& d, cudaStream_t s);
void launch_kick_drift(const Dev& d, int couple, cudaStream_t s);
void launch_clear_wall_history(const Dev& d, int sample, int wall, cudaStream_t s);
void launch_kick_final(const Dev& d, cudaStream_t s);
void launch_cube_after_mid(const Dev& d, cudaStream_t s);
void launch_init(const Dev& d, cudaStream_t s);
void launch_init_check(const Dev& d, cudaStream_t s);
void launch_fp64_math_check(const double* x, int64_t n, double* out, cudaStream_t s);
void launch_gather_state(const Dev& d, cudaStream_t s);
void launch_collect_contacts(const Dev& d, uint32_t* out, unsigned long long cap, cudaStream_t s);
void launch_fluid_mark(const Dev& d, cudaStream_t s);
void launch_fluid_head(const Dev& d, cudaGraphConditionalHandle h, cudaStream_t s);
void launch_fluid_iteration(const Dev& d, cudaGraphConditionalHandle h, cudaStream_t s);
void launch_fluid_tail(const Dev& d, cudaStream_t s);
void launch_react_clear(const Dev& d, cudaStream_t s);
int fluid_blocks(int Cf_total);
int fluid_coop_blocks(int Cf_total);
cudaError_t launch_fluid_solve_coop(const Dev& d, cudaStream_t s);
void launch_collect_springs(const Dev& d, uint32_t* out, double* xi, unsigned long long cap, cudaStream_t s);
void launch_diag(const Dev& d, double* part, cudaStream_t s);
void launch_closure_set(const Dev& d, int enable, int record, cudaStream_t s);
void launch_closure_gather(const Dev& d, cudaStream_t s);
void launch_closure_pack(const float* theta, const float* lo, const float* hi, float cd_max, float cg_max,
                         uint8_t* blob, cudaStream_t s);
}  // namespace cgdem

using namespace cgdem;

// One captured part of cgdem_step: the executable graph, the kernels it
// launches on every replay, and the kernels of a rebuild body it holds.
struct StepGraph {
  cudaGraphExec_t exec = nullptr;
  int kernels = 0;
  int body_kernels = 0;
};
constexpr int GRAPH_HEAD = -1;
constexpr int GRAPH_TAIL = -2;
constexpr int GRAPH_FLUID = -3;  // a Darcy solve on its own (the coupling verbs)

struct cgdem_ctx {
  cgdem_config cfg;
  std::vector<cgdem_sample_params> sp;
  std::vector<SampleDev> sd;
  std::vector<int64_t> counts;
  Dev d;
  double* diag_part = nullptr;
  size_t contact_cap = 0;  // pairs that fit the collection buffer
  bool any_cube = false;
  bool initialised = false;
  std::string err;
  // CUDA graphs of cgdem_step, keyed by (stream, part): part > 0 is a block
  // of that many fused steps, GRAPH_HEAD the opening half kick and drift,
  // GRAPH_TAIL the closing step
  std::map<std::pair<cudaStream_t, int>, StepGraph> graphs;
  bool conditional_graphs = true;
  // kernels that cgdem_step calls launched unconditionally, and the kernels
  // of one candidate-list rebuild sequence (run by a conditional graph node)
  int64_t step_kernels = 0;
  int rebuild_kernels = 0;
};

namespace {

constexpr double PI = 3.14159265358979323846;
constexpr int DIAG_BLOCKS = 128;

int fail(cgdem_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return code;
}

int cuda_fail(cgdem_ctx* c, cudaError_t e, const char* what) {
  return fail(c, CGDEM_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                            \
  do {                                                      \
    cudaError_t e__ = (call);                               \
    if (e__ != cudaSuccess) return cuda_fail(ctx, e__, #call); \
  } while (0)

// Layout of the workspace: a bump allocator with 256-byte alignment.
struct Carver {
  char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

// Derive the device constants of one sample (grain level).
// Separation at which a bonded pair of reduced radius Rs lets go: |delta_C|
// (Table 1, modified JKR) or |delta_S| (point S, original JKR).
double jkr_reach(double gamma, double Es, double Rs, int jkr_mode) {
  const double c = jkr_mode == 1 ? 1.1905507889761495 : 0.5723571212766659;
  return c * std::cbrt(PI * PI * gamma * gamma * Rs / (Es * Es));
}

int derive_sample(cgdem_ctx* ctx, const cgdem_config* cfg, const cgdem_sample_params& p,
                  int64_t first, int64_t count, int cell_off, int fcell_off, SampleDev* out,
                  int* ncells, int* nfcells) {
  SampleDev s;
  memset(&s, 0, sizeof s);
  if (!(p.dt > 0) || !(p.E > 0) || !(p.rho > 0) || !(p.nu > -1 && p.nu < 0.5) ||
      !(p.e > 0 && p.e <= 1) || !(p.mu >= 0) || !(p.gamma >= 0) || !(p.r_max > 0) ||
      !(p.skin > 0) || p.couple_every < 1 || !(p.V_cell > 0) || !(p.n_min > 0 && p.n_min <= 1))
    return fail(ctx, CGDEM_E_INVALID, "sample %lld: a material, time-step or grid parameter is out of range",
                (long long)first);
  for (int k = 0; k < 3; ++k)
    if (p.nf[k] < 1 || !(p.inv_hf[k] > 0) || !(p.hf[k] > 0))
      return fail(ctx, CGDEM_E_INVALID, "fluid grid dimensions must be positive");
  double k_cg = (p.cg_scheme == CGDEM_CG_NONE) ? 1.0 : p.k_cg;
  if (!(k_cg >= 1.0)) return fail(ctx, CGDEM_E_INVALID, "coarse-grain factor k must be >= 1");
  // Eq. 24: gamma_g = k gamma_p; Eq. 19, 28, 34, 35: the rest unchanged.
  s.gamma = k_cg * p.gamma;
  s.rho = p.rho;
  s.Es = p.E / (2.0 * (1.0 - p.nu * p.nu));  // Eq. 12 definitions, equal materials
  {
    double G = p.E / (2.0 * (1.0 + p.nu));
    s.Gs = G / (2.0 * (2.0 - p.nu));  // Mindlin
  }
  {
    double l = std::log(p.e);
    s.beta = -l / std::sqrt(l * l + PI * PI);  // Eq. 33 with ln^2 e
  }
  s.mu = p.mu;
  s.dt = p.dt;
  s.half_dt = 0.5 * p.dt;
  for (int k = 0; k < 3; ++k) s.g[k] = p.g[k];
  s.rho_f = p.rho_f;
  s.mu_f = p.mu_f;
  s.use_drag = p.use_drag;
  s.use_buoyancy = p.use_buoyancy;
  s.kind = p.kind;
  s.coulomb_mode = p.coulomb_mode;
  for (int k = 0; k < 3; ++k) s.L[k] = p.L[k];
  s.Rc = p.Rc;
  s.H = p.H;
  s.r_out = p.r_out;
  const double reach = 2.0 * p.r_max + p.skin;  // largest candidate distance
  // bonded pairs must stay candidates: |delta_C| (modified JKR) or |delta_S|
  // (original JKR) of the largest pair < skin / 2
  if (p.jkr_mode != 0 && p.jkr_mode != 1) return fail(ctx, CGDEM_E_INVALID, "jkr_mode must be 0 or 1");
  s.jkr_mode = p.jkr_mode;
  s.r_max = p.r_max;
  {
    const double dC = jkr_reach(s.gamma, s.Es, 0.5 * p.r_max, p.jkr_mode);
    if (!(2.0 * dC < p.skin))
      return fail(ctx, CGDEM_E_INVALID, "skin %.3g must exceed twice the bond-break separation %.3g",
                  p.skin, dC);
  }
  if (p.kind == CGDEM_PERIODIC_BOX) {
    if (!(p.L[0] > 0) || p.L[0] != p.L[1] || p.L[0] != p.L[2])
      return fail(ctx, CGDEM_E_INVALID, "periodic samples must be cubes");
    if (!(reach < 0.5 * p.L[0]))
      return fail(ctx, CGDEM_E_INVALID, "periodic box too small for 2 r_max + skin");
    s.dq = p.L[0] / 4294967296.0;  // 2^32 steps per period: wrap-around is the minimum image
    s.q_exp = 0x7fffffff;
  } else if (p.kind == CGDEM_CYLINDER) {
    if (!(p.Rc > 0) || !(p.H > 0) || !(p.r_out >= 0))
      return fail(ctx, CGDEM_E_INVALID, "cylinder needs Rc > 0, H > 0, r_out >= 0");
    int e = (int)std::ceil(std::log2(reach / 1073741824.0));  // reach < 2^30 steps
    s.dq = std::ldexp(1.0, e);
    s.q_exp = e;
  } else {
    return fail(ctx, CGDEM_E_INVALID, "unknown domain kind %d", p.kind);
  }
  s.inv_dq = 1.0 / s.dq;
  s.skin_q = (int32_t)std::ceil(p.skin * s.inv_dq) + 8;
  // search grid: each pair is searched from its larger sphere over a stencil
  // of ceil((2R + skin) / h) cells, so h can follow the typical sphere
  const double cs = cfg->cell_scale > 0 ? std::min(1.0, std::max(0.05, cfg->cell_scale)) : 0.35;
  const double h = cs * reach;
  double lo[3], ext[3];
  if (p.kind == CGDEM_PERIODIC_BOX) {
    for (int k = 0; k < 3; ++k) {
      lo[k] = 0.0;
      ext[k] = p.L[k];
    }
  } else {
    lo[0] = lo[1] = -p.Rc;
    ext[0] = ext[1] = 2.0 * p.Rc;
    lo[2] = -4.0 * p.r_max;
    ext[2] = p.H + 4.0 * p.r_max;
  }
  long long ncell = 1;
  for (int k = 0; k < 3; ++k) {
    int n = (int)std::floor(ext[k] / h);
    if (n < 1) n = 1;
    if (n > 1024) n = 1024;
    s.nc[k] = n;
    s.c_lo[k] = lo[k];
    s.c_inv_h[k] = n / ext[k];
    s.c_inv_h_f[k] = (float)s.c_inv_h[k];
    ncell *= n;
  }
  if (ncell > (1ll << 28)) return fail(ctx, CGDEM_E_INVALID, "search grid too large");
  s.cell_off = cell_off;
  *ncells = (int)ncell;
  for (int k = 0; k < 3; ++k) {
    s.nf[k] = p.nf[k];
    s.f_lo[k] = p.f_lo[k];
    s.inv_hf[k] = p.inv_hf[k];
    s.hf[k] = p.hf[k];
  }
  s.fcell_off = fcell_off;
  *nfcells = p.nf[0] * p.nf[1] * p.nf[2];
  s.inv_q = 1099511627776.0 / p.V_cell;  // 2^40 / V_cell
  s.n_min = p.n_min;
  s.vf_mode = p.vf_mode;
  s.couple_every = p.couple_every;
  s.skin = p.skin;
  s.skin_f = (float)p.skin;
  s.rebuild_disp = p.skin - 16.0 * s.dq;
  {
    const double half = 0.5 * (p.skin - 16.0 * s.dq) / s.dq;  // displacement limit, fixed units
    s.rebuild_q2 = (float)(half * half);
  }
  for (int k = 0; k < 3; ++k) {
    s.f_lo_f[k] = (float)p.f_lo[k];
    s.inv_hf_f[k] = (float)p.inv_hf[k];
    s.L_f[k] = (float)p.L[k];
  }
  s.Rc_f = (float)p.Rc;
  s.H_f = (float)p.H;
  s.r_out_f = (float)p.r_out;
  s.first = first;
  s.count = count;
  s.Es_f = (float)s.Es;
  s.Gs_f = (float)s.Gs;
  s.beta_f = (float)s.beta;
  s.mu_f32 = (float)s.mu;
  s.gamma_f = (float)s.gamma;
  s.dt_f = (float)s.dt;
  s.dq_f = (float)s.dq;
  s.rho_f32 = (float)s.rho_f;
  s.muf_f32 = (float)s.mu_f;
  s.n_min_f = (float)s.n_min;
  for (int k = 0; k < 3; ++k) s.g_f[k] = (float)s.g[k];
  s.rho_s_f = (float)s.rho;
  s.k_feat_f = (float)k_cg;
  s.k_cg = k_cg;
  if (p.fluid_mode != 0 && p.fluid_mode != 1)
    return fail(ctx, CGDEM_E_INVALID, "fluid_mode must be 0 or 1");
  if (p.fluid_mode == 1 && (p.kind != CGDEM_CYLINDER || !(p.perm_d > 0) || !std::isfinite(p.p_inlet) ||
                            !p.use_drag))
    return fail(ctx, CGDEM_E_INVALID, "Darcy flow (fluid_mode 1) needs a cylinder, use_drag, perm_d > 0 "
                "and a finite p_inlet");
  s.fluid_mode = p.fluid_mode;
  s.p_inlet = p.p_inlet;
  s.perm_d2 = p.perm_d * p.perm_d / 180.0;
  s.n_psd = 0;  // no size classes until cgdem_set_psd_classes
  // mass quantum: 2^-40 of the largest grain's mass (a grain's quanta fit
  // 40 bits, 2^23 of the largest grains fit a class sum)
  s.psd_mq = std::ldexp(p.rho * (4.0 / 3.0 * PI) * p.r_max * p.r_max * p.r_max, -40);
  {
    const double cd = 2.0 * std::sqrt(5.0 / 6.0);
    s.cdbn = cd * s.beta * std::sqrt(2.0 * s.Es);
    s.cdbt = cd * s.beta * std::sqrt(8.0 * s.Gs);
    s.cdbn_f = (float)s.cdbn;
    s.cdbt_f = (float)s.cdbt;
    s.inv_Es = 1.0 / s.Es;
  }
  *out = s;
  return CGDEM_OK;
}

// Compute (and, with a base pointer, assign) the workspace layout.
int layout(cgdem_ctx* ctx, const cgdem_config* cfg, const cgdem_sample_params* sp,
           const int64_t* counts, char* base, size_t* bytes, std::vector<SampleDev>* sd, Dev* dv,
           double** diag_part, size_t* contact_cap, bool* any_cube) {
  if (!cfg || !sp || !counts || cfg->n_samples < 1)
    return fail(ctx, CGDEM_E_INVALID, "null argument or n_samples < 1");
  if (cfg->precision != CGDEM_FP64 && cfg->precision != CGDEM_MIXED)
    return fail(ctx, CGDEM_E_INVALID, "unknown precision");
  if (cfg->closure != 0 && cfg->closure != 1) return fail(ctx, CGDEM_E_INVALID, "closure must be 0 or 1");
  if (cfg->particles_per_warp != 0 && cfg->particles_per_warp != 16 && cfg->particles_per_warp != 32)
    return fail(ctx, CGDEM_E_INVALID, "particles_per_warp must be 0, 16 or 32");
  if (cfg->fluid_kernels != 0 && cfg->fluid_kernels != 1)
    return fail(ctx, CGDEM_E_INVALID, "fluid_kernels must be 0 or 1");
  for (int k = 0; k < cfg->n_samples; ++k)
    if (cfg->closure && sp[k].jkr_mode == 1)
      return fail(ctx, CGDEM_E_INVALID, "the original JKR runs in contexts without the learned closure");
  if (cfg->closure && cfg->block_size != 128 && cfg->block_size > 0)
    return fail(ctx, CGDEM_E_INVALID, "a context with the learned closure runs blocks of 128 threads");
  const int S = cfg->n_samples;
  int64_t N = 0;
  int C = 0, Cf = 0;
  bool cyl = false, cube = false;
  sd->resize(S);
  for (int s = 0; s < S; ++s) {
    if (counts[s] < 0) return fail(ctx, CGDEM_E_INVALID, "negative particle count");
    if (sp[s].couple_every != sp[0].couple_every)
      return fail(ctx, CGDEM_E_INVALID, "couple_every must be equal in all samples");
    int nc = 0, nfc = 0;
    int r = derive_sample(ctx, cfg, sp[s], N, counts[s], C, Cf, &(*sd)[s], &nc, &nfc);
    if (r) return r;
    N += counts[s];
    C += nc;
    Cf += nfc;
    cyl |= sp[s].kind == CGDEM_CYLINDER;
    cube |= sp[s].vf_mode == 1;
  }
  if (N >= (1ll << 30)) return fail(ctx, CGDEM_E_INVALID, "too many particles");
  const int cap = cfg->max_neighbors > 0 ? cfg->max_neighbors : 48;
  if (cap > CGDEM_MAX_NEIGHBORS)
    return fail(ctx, CGDEM_E_INVALID, "max_neighbors must be <= %d", CGDEM_MAX_NEIGHBORS);
  // a multiple of every block size used, so grids over Npad never run past it
  const int Npad = (int)(((N + 255) / 256) * 256 + 256);
  const bool mixed = cfg->precision == CGDEM_MIXED;
  Carver cv{base};
  Dev d;
  memset(&d, 0, sizeof d);
  for (int b = 0; b < 2; ++b) {
    d.pos[b] = cv.take<double4>(Npad);
    d.vel[b] = cv.take<double4>(Npad);
    d.omg[b] = cv.take<double4>(Npad);
    d.posq[b] = cv.take<int4>(Npad);
    d.velf[b] = cv.take<float4>(Npad);
    d.omgf[b] = cv.take<float4>(Npad);
    d.id[b] = cv.take<int>(Npad);
    d.sample[b] = cv.take<int>(Npad);
    d.fcell[b] = cv.take<int>(Npad);
    d.vq[b] = cv.take<unsigned long long>(Npad);
    if (cyl) {
      if (mixed) d.wallhf[b] = cv.take<float4>(CGDEM_WALLS * (size_t)Npad);
      else d.wallh[b] = cv.take<double4>(CGDEM_WALLS * (size_t)Npad);
    }
    d.rec[b] = mixed ? (void*)cv.take<RecF>((size_t)cap * Npad) : (void*)cv.take<RecD>((size_t)cap * Npad);
    d.cnt[b] = cv.take<uint32_t>(Npad);
    d.roff[b] = cv.take<uint32_t>(Npad);
  }
  d.posq_ref = cv.take<int4>(Npad);
  if (mixed) d.sched = cv.take<uint32_t>(Npad);
  if (!mixed) {  // pairs listed once
    d.inc = cv.take<uint32_t>((size_t)cap * Npad);
    d.inc_n = cv.take<uint32_t>(Npad);
    d.rslot = cv.take<uint32_t>((size_t)cap * Npad);
    d.inbox = cv.take<double4>(2 * (size_t)cap * Npad);
    d.seg_flag = cv.take<uint32_t>(Npad / 16);
    d.seg_wait = cv.take<uint32_t>(Npad / 16);
    if (cfg->closure) d.inbox_cl = cv.take<float4>((size_t)cap * Npad);
  }
  d.cand_tmp = cv.take<uint32_t>((size_t)cap * Npad);
  d.cand_n = cv.take<uint32_t>(Npad);
  d.big_list = cv.take<uint32_t>(Npad);
  d.big_n = cv.take<uint32_t>(1);
  d.tile_sums = cv.take<uint32_t>((size_t)(C + 2) / 2048 + 2);
  d.dmax2 = cv.take<unsigned>(S);
  d.F = cv.take<double4>(Npad);
  d.T = cv.take<double4>(Npad);
  d.cell_count = cv.take<uint32_t>((size_t)C + 2);
  d.cell_start = cv.take<uint32_t>((size_t)C + 2);
  d.pcell = cv.take<uint32_t>(Npad);
  d.pslot = cv.take<uint32_t>(Npad);
  d.perm_tmp = cv.take<uint32_t>(Npad);
  d.perm = cv.take<uint32_t>(Npad);
  d.inv_perm = cv.take<uint32_t>(Npad);
  for (int b = 0; b < 3; ++b) d.vf[b] = cv.take<unsigned long long>((size_t)Cf + 1);
  d.Us = cv.take<double4>((size_t)Cf + 1);
  d.Usf = cv.take<float4>((size_t)Cf + 1);
  d.removed_step = cv.take<int>(Npad);
  d.disp = cv.take<double>(S);
  d.vmax2 = cv.take<unsigned long long>(S);
  d.diag = cv.take<double>(8 * (size_t)S);
  d.stage = cv.take<StageDev>(S);
  bool fluid = false;
  for (int k = 0; k < S; ++k) fluid |= sp[k].fluid_mode == 1;
  if (fluid) {
    const size_t nc = (size_t)Cf + 1;
    d.fl_sample = cv.take<int>(nc);
    d.fl_type = cv.take<signed char>(nc);
    d.fl_K = cv.take<double>(nc);
    d.fl_p = cv.take<double>(nc);
    d.fl_r = cv.take<double>(nc);
    d.fl_z = cv.take<double>(nc);
    d.fl_d = cv.take<double>(nc);
    d.fl_q = cv.take<double>(nc);
    d.fl_M = cv.take<double>(nc);
    d.fl_b = cv.take<double>(nc);
    d.fl_d2 = cv.take<double>(nc);
    d.fl_T = cv.take<double4>(nc);
    d.fl_blocks = fluid_blocks(Cf);
    d.fl_part = cv.take<double>(4 * (size_t)d.fl_blocks);
    d.gradp = cv.take<double4>(nc);
    d.gradpf = cv.take<float4>(nc);
    d.react[0] = cv.take<unsigned long long>(3 * nc);
    d.react[1] = cv.take<unsigned long long>(3 * nc);
    d.any_fluid = 1;
  }
  d.fl_iters_max = cfg->fluid_iters > 0 ? cfg->fluid_iters : 2000;
  d.fl_tol = cfg->fluid_tol > 0 ? cfg->fluid_tol : 1e-10;
  d.psd_count = cv.take<unsigned long long>((size_t)CGDEM_PSD_MAX * S);
  d.psd_mass = cv.take<unsigned long long>((size_t)CGDEM_PSD_MAX * S);
  d.staging = cv.take<double>(16 * (size_t)Npad);
  d.contact_n = cv.take<unsigned long long>(1);
  if (cfg->closure) {
    d.clc[0] = cv.take<float2>(Npad);
    d.clc[1] = cv.take<float2>(Npad);
    d.clrec = cv.take<float>((size_t)CL_COLS * Npad);
    d.clblob = cv.take<uint8_t>(CL_BLOB);
  }
  d.sp = cv.take<SampleDev>(S);
  d.ctl = cv.take<Ctl>(1);
  *diag_part = cv.take<double>((size_t)DIAG_BLOCKS * 8 * S);
  // collected contacts reuse the spare record buffer
  const size_t rec_bytes = (size_t)cap * Npad * (mixed ? sizeof(RecF) : sizeof(RecD));
  *contact_cap = rec_bytes / 8;
  d.N = (int)N;
  d.Npad = Npad;
  d.cap = cap;
  d.n_samples = S;
  d.C_total = C;
  d.Cf_total = Cf;
  d.mixed = mixed ? 1 : 0;
  d.ppw = cfg->particles_per_warp == 16 ? 16 : 32;
  d.rstride = mixed ? d.ppw : 1;
  *bytes = cv.off + 256;
  *dv = d;
  *any_cube = cube;
  return CGDEM_OK;
}

cudaStream_t st(void* s) { return reinterpret_cast<cudaStream_t>(s); }

int check_status(cgdem_ctx* ctx, cudaStream_t s) {
  Ctl c;
  CK(cudaMemcpyAsync(&c, ctx->d.ctl, sizeof c, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (c.status & ST_CAPACITY)
    return fail(ctx, CGDEM_E_CAPACITY, "a particle had %d candidates; max_neighbors is %d", c.max_cand,
                ctx->d.cap);
  if (c.status & ST_BOND_LOST)
    return fail(ctx, CGDEM_E_STATE,
                "a bonded pair left the candidate list (skin too small): particles %d and %d, squared "
                "distance %llu vs squared reach %llu (fixed-point units)",
                c.lost_i, c.lost_j, c.lost_d2, c.lost_S2);
  if (c.status & ST_NONFINITE) return fail(ctx, CGDEM_E_NONFINITE, "a force became NaN or Inf");
  if (c.status & ST_TIMEOUT)
    return fail(ctx, CGDEM_E_TIMEOUT, "a bounded wait of the closure network expired (corrections reset to 1)");
  return CGDEM_OK;
}

int ready(cgdem_ctx* ctx) {
  if (!ctx) return CGDEM_E_INVALID;
  if (!ctx->initialised) return fail(ctx, CGDEM_E_STATE, "cgdem_init_particles has not been called");
  return CGDEM_OK;
}

// Kernel nodes of a graph (the bodies of conditional nodes are not counted).
int count_kernels(cudaGraph_t g) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return 0;
  std::vector<cudaGraphNode_t> nodes(n);
  if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
  int k = 0;
  for (size_t i = 0; i < n; ++i) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

// Append to the capture on cs a conditional (IF) node whose body is the
// rebuild sequence, captured on bs; its condition is handle h.
cudaError_t add_rebuild_node(cgdem_ctx* ctx, cudaStream_t cs, cudaStream_t bs,
                             cudaGraphConditionalHandle h, int* body_kernels) {
  cudaStreamCaptureStatus stt;
  cudaGraph_t cg;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(cs, &stt, nullptr, &cg, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeIf;
  cp.conditional.size = 1;
  cudaGraphNode_t cn;
  e = cudaGraphAddNode(&cn, cg, deps, nullptr, nd, &cp);
  if (e != cudaSuccess) return e;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  launch_rebuild(ctx->d, bs);
  e = cudaStreamEndCapture(bs, &body);
  if (e != cudaSuccess) return e;
  *body_kernels = count_kernels(body);
  return cudaStreamUpdateCaptureDependencies(cs, &cn, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// Append to the capture on cs a conditional (IF) node whose body, captured
// on bs, is the one-launch Darcy solve; its condition is handle h, which the
// step's force kernel sets when the step updated the porosity.
cudaError_t add_fluid_if(cgdem_ctx* ctx, cudaStream_t cs, cudaStream_t bs, cudaGraphConditionalHandle h) {
  cudaStreamCaptureStatus stt;
  cudaGraph_t cg;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(cs, &stt, nullptr, &cg, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeIf;
  cp.conditional.size = 1;
  cudaGraphNode_t cn;
  e = cudaGraphAddNode(&cn, cg, deps, nullptr, nd, &cp);
  if (e != cudaSuccess) return e;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  e = launch_fluid_solve_coop(ctx->d, bs);
  cudaError_t e2 = cudaStreamEndCapture(bs, &body);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return e;
  return cudaStreamUpdateCaptureDependencies(cs, &cn, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// Append a Darcy solve to the capture on cs (it does nothing unless a
// porosity update is pending): the set-up kernels, then the conjugate-gradient
// iterations as the body of a WHILE node (captured on bs) whose condition the
// kernels set, then the velocity field.  Without conditional nodes, the
// iterations are captured fluid_iters times (each returns at once once the
// solve has converged).
cudaError_t add_fluid_solve(cgdem_ctx* ctx, cudaStream_t cs, cudaStream_t bs, bool conditional) {
  if (ctx->d.fl_coop_blocks > 0) return launch_fluid_solve_coop(ctx->d, cs);
  if (!conditional) {
    launch_fluid_head(ctx->d, 0, cs);
    for (int i = 0; i < ctx->d.fl_iters_max; ++i) launch_fluid_iteration(ctx->d, 0, cs);
    launch_fluid_tail(ctx->d, cs);
    return cudaSuccess;
  }
  cudaStreamCaptureStatus stt;
  cudaGraph_t cg;
  cudaError_t e = cudaStreamGetCaptureInfo(cs, &stt, nullptr, &cg, nullptr, nullptr, nullptr);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, cg, 0u, 0u);
  if (e != cudaSuccess) return e;
  launch_fluid_head(ctx->d, h, cs);
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  e = cudaStreamGetCaptureInfo(cs, &stt, nullptr, &cg, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cn;
  e = cudaGraphAddNode(&cn, cg, deps, nullptr, nd, &cp);
  if (e != cudaSuccess) return e;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  launch_fluid_iteration(ctx->d, h, bs);
  e = cudaStreamEndCapture(bs, &body);
  if (e != cudaSuccess) return e;
  e = cudaStreamUpdateCaptureDependencies(cs, &cn, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) return e;
  launch_fluid_tail(ctx->d, cs);
  return cudaSuccess;
}

// Capture one part of cgdem_step into a graph:
//   part = U > 0: U fused steps (rebuild if flagged, forces, kick, drift,
//     porosity).  Each step's rebuild sequence sits in the body of a
//     conditional (IF) node whose condition the previous step's force kernel
//     sets from the device-side rebuild flag (the first step's, a one-thread
//     kernel at the graph's start), so a step without a rebuild launches one
//     kernel;
//   GRAPH_HEAD: the half kick and drift that open a call (state at a full
//     step -> the first mid-step state);
//   GRAPH_TAIL: the closing step, which ends on the full-step state (forces,
//     v(n), w(n)): conditional rebuild, then the force evaluation.
// Without conditional nodes the rebuild kernels are captured plainly (they
// return at once unless a rebuild is due).
cudaError_t capture_part(cgdem_ctx* ctx, int part, bool conditional, StepGraph* out) {
  cudaStream_t cs, bs;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return e;
  }
  cudaGraph_t g = nullptr;
  int body_kernels = 0;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (part == GRAPH_HEAD || part == GRAPH_FLUID) {
    if (e == cudaSuccess && part == GRAPH_HEAD) launch_kick_drift(ctx->d, 1, cs);
    if (e == cudaSuccess && ctx->d.any_fluid) e = add_fluid_solve(ctx, cs, bs, conditional);
  } else {
    const int U = part > 0 ? part : 1;
    const bool tail = part == GRAPH_TAIL;
    // one handle per step: a one-thread kernel sets the first from the device
    // flag at every launch of the graph; step i's force kernel sets step i + 1's
    std::vector<cudaGraphConditionalHandle> hs;
    // with the one-launch Darcy solve, each step's solve sits in an IF node
    // that the step's force kernel sets (nothing launches on the steps that
    // do not update the porosity)
    const bool fluid_if = conditional && !tail && ctx->d.any_fluid && ctx->d.fl_coop_blocks > 0;
    std::vector<cudaGraphConditionalHandle> hf;
    if (conditional && e == cudaSuccess) {
      cudaStreamCaptureStatus stt;
      cudaGraph_t cg;
      e = cudaStreamGetCaptureInfo(cs, &stt, nullptr, &cg, nullptr, nullptr, nullptr);
      hs.resize(U);
      for (int i = 0; i < U && e == cudaSuccess; ++i)
        e = cudaGraphConditionalHandleCreate(&hs[i], cg, i == 0 ? 1u : 0u,
                                             i == 0 ? cudaGraphCondAssignDefault : 0u);
      if (fluid_if) {
        hf.resize(U);
        for (int i = 0; i < U && e == cudaSuccess; ++i)
          e = cudaGraphConditionalHandleCreate(&hf[i], cg, 0u, cudaGraphCondAssignDefault);
      }
    }
    for (int i = 0; i < U && e == cudaSuccess; ++i) {
      if (conditional) {
        if (i == 0) launch_rebuild_cond(ctx->d, hs[0], cs);
        e = add_rebuild_node(ctx, cs, bs, hs[i], &body_kernels);
        if (e != cudaSuccess) break;
      } else {
        launch_rebuild(ctx->d, cs);
      }
      if (tail) {
        launch_forces(ctx->d, 2, ctx->cfg.block_size, cs, 0);
      } else {
        launch_forces(ctx->d, 1, ctx->cfg.block_size, cs,
                      conditional && i + 1 < U ? hs[i + 1] : 0, fluid_if ? hf[i] : 0);
        if (ctx->any_cube) launch_cube_after_mid(ctx->d, cs);
        if (fluid_if) {
          e = add_fluid_if(ctx, cs, bs, hf[i]);
          if (e != cudaSuccess) break;
        } else if (ctx->d.any_fluid) {
          e = add_fluid_solve(ctx, cs, bs, conditional);
          if (e != cudaSuccess) break;
        }
      }
    }
  }
  cudaError_t e2 = cudaStreamEndCapture(cs, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) {
    out->kernels = count_kernels(g);
    out->body_kernels = body_kernels;
    e = cudaGraphInstantiate(&out->exec, g, 0);
  }
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  cudaStreamDestroy(bs);
  cudaGetLastError();  // a failed attempt must not leave a sticky launch error behind
  return e;
}

void drop_graphs(cgdem_ctx* ctx) {
  for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second.exec);
  ctx->graphs.clear();
}

// The captured graph of one part of cgdem_step for stream s (captured on
// first use for this stream).
int find_part(cgdem_ctx* ctx, int part, cudaStream_t s, StepGraph** out) {
  const auto key = std::make_pair(s, part);
  auto it = ctx->graphs.find(key);
  if (it == ctx->graphs.end()) {
    StepGraph g;
    cudaError_t e = cudaErrorUnknown;
    if (ctx->conditional_graphs) {
      e = capture_part(ctx, part, true, &g);
      if (e != cudaSuccess && ctx->d.fl_coop_blocks > 0) {
        // no cooperative launch in a graph: the Darcy solve as separate kernels from now on
        ctx->d.fl_coop_blocks = 0;
        drop_graphs(ctx);
        e = capture_part(ctx, part, true, &g);
      }
      if (e != cudaSuccess) {  // conditional nodes unavailable: plain captures from now on
        ctx->conditional_graphs = false;
        drop_graphs(ctx);
      }
    }
    if (e != cudaSuccess) e = capture_part(ctx, part, false, &g);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "graph capture");
    // upload now, so that the first replay does not pay it
    CK(cudaGraphUpload(g.exec, s));
    it = ctx->graphs.emplace(key, g).first;
  }
  *out = &it->second;
  return CGDEM_OK;
}

// Launch part of cgdem_step on s.
int launch_part(cgdem_ctx* ctx, int part, cudaStream_t s) {
  StepGraph* g = nullptr;
  int r = find_part(ctx, part, s, &g);
  if (r) return r;
  CK(cudaGraphLaunch(g->exec, s));
  if (part != GRAPH_FLUID) ctx->step_kernels += g->kernels;
  if (g->body_kernels) ctx->rebuild_kernels = g->body_kernels;
  return CGDEM_OK;
}

// Capture every part that cgdem_step may launch on s (the opening and
// closing parts, U steps and each power of two below U), so that the first
// call on a stream pays all captures and later calls of any length replay.
int prepare_parts(cgdem_ctx* ctx, cudaStream_t s) {
  if (ctx->graphs.count(std::make_pair(s, GRAPH_HEAD))) return CGDEM_OK;
  StepGraph* g = nullptr;
  int r;
  if ((r = find_part(ctx, GRAPH_TAIL, s, &g))) return r;
  const int U = ctx->cfg.steps_per_graph;
  if ((r = find_part(ctx, U, s, &g))) return r;
  for (int b = 1 << 30; b >= 1; b >>= 1)
    if (b < U && (r = find_part(ctx, b, s, &g))) return r;
  return find_part(ctx, GRAPH_HEAD, s, &g);
}

}  // namespace

extern "C" {

double cgdem_rayleigh_dt(double Rbar, double rho, double E, double nu) {
  // Eq. 37-38, shear modulus G = E / (2 (1 + nu))
  const double G = E / (2.0 * (1.0 + nu));
  const double beta = 0.8766 + 0.163 * nu;
  return PI * Rbar / beta * std::sqrt(rho / G);
}

int cgdem_cg_scale_diameters(const double* d_fine, int64_t n_fine, double k, int scheme,
                             double* d_out, int64_t* n_out) {
  if (!d_fine || !d_out || !n_out || n_fine < 0 || !(k >= 1.0)) return CGDEM_E_INVALID;
  if (scheme == CGDEM_CG_NONE || k == 1.0) {
    std::memcpy(d_out, d_fine, sizeof(double) * (size_t)n_fine);
    *n_out = n_fine;
    return CGDEM_OK;
  }
  // Eq. 15-16: n_CG = k^3 fine particles per grain
  const int64_t ng = (int64_t)std::floor((double)n_fine / (k * k * k) + 1e-9);
  if (scheme == CGDEM_CG_SSW) {  // Eq. 14 per particle: PSD shape kept
    for (int64_t i = 0; i < ng; ++i) d_out[i] = k * d_fine[i];
  } else if (scheme == CGDEM_CG_SSP) {  // one size: k times the volume-mean diameter
    long double acc = 0;
    for (int64_t i = 0; i < n_fine; ++i) acc += (long double)d_fine[i] * d_fine[i] * d_fine[i];
    const double dbar = std::cbrt((double)(acc / (long double)n_fine));
    for (int64_t i = 0; i < ng; ++i) d_out[i] = k * dbar;
  } else {
    return CGDEM_E_INVALID;
  }
  *n_out = ng;
  return CGDEM_OK;
}

int cgdem_workspace_size(const cgdem_config* cfg, const cgdem_sample_params* sp,
                         const int64_t* counts, size_t* bytes) {
  if (!bytes) return CGDEM_E_INVALID;
  std::vector<SampleDev> sd;
  Dev d;
  double* dp;
  size_t cc;
  bool cube;
  return layout(nullptr, cfg, sp, counts, nullptr, bytes, &sd, &d, &dp, &cc, &cube);
}

int cgdem_create(const cgdem_config* cfg, const cgdem_sample_params* sp, const int64_t* counts,
                 void* workspace, size_t bytes, cgdem_ctx** out) {
  if (!out) return CGDEM_E_INVALID;
  *out = nullptr;
  cgdem_ctx* ctx = new cgdem_ctx();
  size_t need = 0;
  int r = layout(ctx, cfg, sp, counts, nullptr, &need, &ctx->sd, &ctx->d, &ctx->diag_part,
                 &ctx->contact_cap, &ctx->any_cube);
  if (r) {
    // keep the message: callers read it through a temporary context
    static thread_local std::string last;
    last = ctx->err;
    delete ctx;
    fprintf(stderr, "cgdem_create: %s\n", last.c_str());
    return r;
  }
  if (!workspace || bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
    fprintf(stderr, "cgdem_create: workspace must be 256-byte aligned and >= %zu bytes\n", need);
    delete ctx;
    return CGDEM_E_INVALID;
  }
  layout(ctx, cfg, sp, counts, reinterpret_cast<char*>(workspace), &need, &ctx->sd, &ctx->d,
         &ctx->diag_part, &ctx->contact_cap, &ctx->any_cube);
  ctx->cfg = *cfg;
  if (ctx->cfg.block_size <= 0) ctx->cfg.block_size = 128;
  if (ctx->cfg.block_size != 64 && ctx->cfg.block_size != 128 && ctx->cfg.block_size != 256) {
    delete ctx;
    return CGDEM_E_INVALID;
  }
  if (ctx->cfg.steps_per_graph <= 0) ctx->cfg.steps_per_graph = 32;
  ctx->sp.assign(sp, sp + cfg->n_samples);
  ctx->counts.assign(counts, counts + cfg->n_samples);
  cudaError_t e = cudaMemcpy(ctx->d.sp, ctx->sd.data(), sizeof(SampleDev) * ctx->sd.size(),
                             cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    fprintf(stderr, "cgdem_create: %s\n", cudaGetErrorString(e));
    delete ctx;
    return CGDEM_E_CUDA;
  }
  // fluid velocity starts at zero
  cudaMemset(ctx->d.Us, 0, sizeof(double4) * ((size_t)ctx->d.Cf_total + 1));
  cudaMemset(ctx->d.Usf, 0, sizeof(float4) * ((size_t)ctx->d.Cf_total + 1));
  if (ctx->d.any_fluid) {  // Darcy flow: each cell's sample; pressures and gradients start at zero
    const size_t nc = (size_t)ctx->d.Cf_total + 1;
    std::vector<int> cs(nc, 0);
    for (size_t k = 0; k < ctx->sd.size(); ++k)
      for (int c = 0; c < ctx->sd[k].nf[0] * ctx->sd[k].nf[1] * ctx->sd[k].nf[2]; ++c)
        cs[(size_t)ctx->sd[k].fcell_off + c] = (int)k;
    cudaMemcpy(ctx->d.fl_sample, cs.data(), sizeof(int) * nc, cudaMemcpyHostToDevice);
    cudaMemset(ctx->d.fl_p, 0, sizeof(double) * nc);
    cudaMemset(ctx->d.fl_type, 2, nc);
    cudaMemset(ctx->d.gradp, 0, sizeof(double4) * nc);
    cudaMemset(ctx->d.gradpf, 0, sizeof(float4) * nc);
    cudaMemset(ctx->d.react[0], 0, sizeof(unsigned long long) * 3 * nc);
    cudaMemset(ctx->d.react[1], 0, sizeof(unsigned long long) * 3 * nc);
    ctx->d.fl_coop_blocks = cfg->fluid_kernels == 1 ? 0 : fluid_coop_blocks(ctx->d.Cf_total);
  }
  for (const auto& q : ctx->sd) ctx->d.prep |= q.jkr_mode == 1 ? 1 : 0;
  {  // preparation stages: the top plate at the sample's H, no penetrometer
    std::vector<StageDev> st(ctx->sd.size());
    for (size_t k = 0; k < st.size(); ++k) {
      st[k] = StageDev{};
      st[k].H = ctx->sd[k].H;
    }
    cudaMemcpy(ctx->d.stage, st.data(), sizeof(StageDev) * st.size(), cudaMemcpyHostToDevice);
  }
  *out = ctx;
  return CGDEM_OK;
}

void cgdem_destroy(cgdem_ctx* ctx) {
  if (!ctx) return;
  drop_graphs(ctx);
  delete ctx;
}

const char* cgdem_last_error(const cgdem_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int cgdem_status_sync(cgdem_ctx* ctx, void* stream) {
  int r = ready(ctx);
  if (r) return r;
  return check_status(ctx, st(stream));
}

int cgdem_set_fluid_velocity(cgdem_ctx* ctx, const double* Us, void* stream) {
  if (!ctx || !Us) return CGDEM_E_INVALID;
  const int Cf = ctx->d.Cf_total;
  std::vector<double4> a((size_t)Cf + 1);
  std::vector<float4> b((size_t)Cf + 1);
  for (int c = 0; c < Cf; ++c) {
    a[c] = make_double4(Us[3 * c], Us[3 * c + 1], Us[3 * c + 2], 0.0);
    b[c] = make_float4((float)Us[3 * c], (float)Us[3 * c + 1], (float)Us[3 * c + 2], 0.f);
  }
  a[Cf] = make_double4(0, 0, 0, 0);
  b[Cf] = make_float4(0, 0, 0, 0);
  cudaStream_t s = st(stream);
  CK(cudaMemcpyAsync(ctx->d.Us, a.data(), sizeof(double4) * a.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ctx->d.Usf, b.data(), sizeof(float4) * b.size(), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  return CGDEM_OK;
}

int cgdem_init_particles(cgdem_ctx* ctx, const double* x, const double* v, const double* w,
                         const double* R, int bond_touching, void* stream) {
  if (!ctx || (!x && ctx->d.N) || (!v && ctx->d.N) || (!w && ctx->d.N) || (!R && ctx->d.N))
    return CGDEM_E_INVALID;
  const size_t N = ctx->d.N;
  cudaStream_t s = st(stream);
  double* stg = ctx->d.staging;
  if (N) {
    CK(cudaMemcpyAsync(stg, x, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(stg + 3 * N, v, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(stg + 6 * N, w, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(stg + 9 * N, R, sizeof(double) * N, cudaMemcpyHostToDevice, s));
    // the inputs are checked on the device, before any kernel bins them: the
    // lowest index with a radius outside (0, r_max], and the lowest with a
    // non-finite position, velocity or angular velocity
    long long* bad = &ctx->d.ctl->init_bad_r;
    CK(cudaMemsetAsync(bad, 0x7f, 2 * sizeof(long long), s));
    launch_init_check(ctx->d, s);
    long long hb[2];
    CK(cudaMemcpyAsync(hb, bad, sizeof hb, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const long long i = std::min(hb[0], hb[1]);
    if (i < (long long)N) {
      if (hb[0] == i)
        return fail(ctx, CGDEM_E_INVALID, "radius of particle %lld outside (0, r_max]", i);
      return fail(ctx, CGDEM_E_NONFINITE, "non-finite state of particle %lld", i);
    }
  }
  launch_init(ctx->d, s);
  for (int b = 0; b < 3; ++b)
    CK(cudaMemsetAsync(ctx->d.vf[b], 0, sizeof(unsigned long long) * ((size_t)ctx->d.Cf_total + 1), s));
  CK(cudaMemsetAsync(ctx->d.cell_count, 0, sizeof(uint32_t) * ((size_t)ctx->d.C_total + 2), s));
  if (ctx->d.seg_flag)
    CK(cudaMemsetAsync(ctx->d.seg_flag, 0, sizeof(uint32_t) * (size_t)(ctx->d.Npad / 16), s));
  CK(cudaMemsetAsync(ctx->d.psd_count, 0, sizeof(unsigned long long) * CGDEM_PSD_MAX * ctx->d.n_samples, s));
  CK(cudaMemsetAsync(ctx->d.psd_mass, 0, sizeof(unsigned long long) * CGDEM_PSD_MAX * ctx->d.n_samples, s));
  launch_set_rebuild(ctx->d, s);
  launch_rebuild(ctx->d, s);
  if (bond_touching) launch_bond_touching(ctx->d, s);
  launch_couple(ctx->d, s);
  if (ctx->d.any_fluid) {  // the initial Darcy flow of the initial porosity
    launch_fluid_mark(ctx->d, s);
    int rr = launch_part(ctx, GRAPH_FLUID, s);
    if (rr) return rr;
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  ctx->initialised = true;
  return check_status(ctx, s);
}

int cgdem_build_contacts(cgdem_ctx* ctx, void* stream) {
  int r = ready(ctx);
  if (r) return r;
  cudaStream_t s = st(stream);
  launch_set_rebuild(ctx->d, s);
  launch_rebuild(ctx->d, s);
  CK(cudaGetLastError());
  return CGDEM_OK;
}

int cgdem_couple_fluid(cgdem_ctx* ctx, void* stream) {
  int r = ready(ctx);
  if (r) return r;
  launch_couple(ctx->d, st(stream));
  if (ctx->d.any_fluid) {  // two-way coupling: the Darcy flow of the new porosity
    launch_fluid_mark(ctx->d, st(stream));
    if ((r = launch_part(ctx, GRAPH_FLUID, st(stream)))) return r;
  }
  CK(cudaGetLastError());
  return CGDEM_OK;
}

int cgdem_compute_forces(cgdem_ctx* ctx, void* stream) {
  int r = ready(ctx);
  if (r) return r;
  if (ctx->d.any_fluid) launch_react_clear(ctx->d, st(stream));
  launch_forces(ctx->d, 0, ctx->cfg.block_size, st(stream), 0);
  CK(cudaGetLastError());
  return CGDEM_OK;
}

int cgdem_integrate(cgdem_ctx* ctx, int half, void* stream) {
  int r = ready(ctx);
  if (r) return r;
  if (half == 0) launch_kick_drift(ctx->d, 0, st(stream));
  else if (half == 1) launch_kick_final(ctx->d, st(stream));
  else return fail(ctx, CGDEM_E_INVALID, "half must be 0 or 1");
  CK(cudaGetLastError());
  return CGDEM_OK;
}

int cgdem_fp64_math_check(const double* x, int64_t n, double* out, void* stream) {
  if (n < 0 || (n > 0 && (!x || !out))) return CGDEM_E_INVALID;
  launch_fp64_math_check(x, n, out, st(stream));
  return cudaGetLastError() == cudaSuccess ? CGDEM_OK : CGDEM_E_CUDA;
}

int cgdem_prepare(cgdem_ctx* ctx, void* stream) {
  if (!ctx) return CGDEM_E_INVALID;
  if (ctx->d.N == 0) return CGDEM_OK;
  return prepare_parts(ctx, st(stream));
}

int cgdem_step(cgdem_ctx* ctx, int64_t nsteps, void* stream) {
  int r = ready(ctx);
  if (r) return r;
  if (nsteps < 0) return fail(ctx, CGDEM_E_INVALID, "nsteps < 0");
  if (nsteps == 0 || ctx->d.N == 0) return CGDEM_OK;
  cudaStream_t s = st(stream);
  if ((r = prepare_parts(ctx, s))) return r;
  // half kick + drift from the full-step state, porosity of the new positions
  if ((r = launch_part(ctx, GRAPH_HEAD, s))) return r;
  // the nsteps - 1 fused steps as graphs of U steps, then of the powers of
  // two below U (each captured once per stream), so that every call runs
  // from graphs whatever its length
  int64_t body = nsteps - 1;
  const int U = ctx->cfg.steps_per_graph;
  while (body >= U) {
    if ((r = launch_part(ctx, U, s))) return r;
    body -= U;
  }
  for (int b = 1 << 30; b >= 1; b >>= 1) {
    if (b >= U || body < b) continue;
    if ((r = launch_part(ctx, b, s))) return r;
    body -= b;
  }
  // last step ends on the full-step state (forces, v(n), w(n))
  return launch_part(ctx, GRAPH_TAIL, s);
}

int cgdem_set_closure(cgdem_ctx* ctx, const float* theta, const cgdem_closure_params* cp, int enable,
                      void* stream) {
  int r = ready(ctx);
  if (r) return r;
  if (!ctx->d.clblob) return fail(ctx, CGDEM_E_STATE, "the context was created without closure support");
  cudaStream_t s = st(stream);
  if (enable) {
    if (!theta || !cp) return fail(ctx, CGDEM_E_INVALID, "enabling the closure needs theta and its parameters");
    if (!(cp->cd_log_max >= 0.f) || !(cp->cg_log_max >= 0.f) || !(cp->cd_log_max <= 20.f) ||
        !(cp->cg_log_max <= 20.f))
      return fail(ctx, CGDEM_E_INVALID, "correction bounds must lie in [0, 20]");
    // bonded pairs must stay candidates at the largest corrected surface energy
    const double cmax = std::exp((double)cp->cg_log_max);
    for (size_t i = 0; i < ctx->sd.size(); ++i) {
      const SampleDev& S = ctx->sd[i];
      const double Rs = 0.5 * ctx->sp[i].r_max, g = S.gamma * cmax;
      const double dC = jkr_reach(g, S.Es, Rs, S.jkr_mode);
      if (!(2.0 * dC < ctx->sp[i].skin))
        return fail(ctx, CGDEM_E_INVALID,
                    "sample %zu: skin %.3g must exceed twice the bond-break separation %.3g at "
                    "the largest surface-energy correction", i, ctx->sp[i].skin, dC);
    }
    launch_closure_pack(theta, cp->lo, cp->hi, cp->cd_log_max, cp->cg_log_max, ctx->d.clblob, s);
  }
  launch_closure_set(ctx->d, enable ? 1 : 0, -1, s);
  CK(cudaGetLastError());
  // the force launches change shape: captured step graphs are rebuilt
  ctx->d.cl_smem = enable ? 1 : 0;
  CK(cudaStreamSynchronize(s));
  drop_graphs(ctx);
  return CGDEM_OK;
}

int cgdem_closure_record(cgdem_ctx* ctx, int enable, void* stream) {
  int r = ready(ctx);
  if (r) return r;
  if (!ctx->d.clblob) return fail(ctx, CGDEM_E_STATE, "the context was created without closure support");
  cudaStream_t s = st(stream);
  launch_closure_set(ctx->d, -1, enable ? 1 : 0, s);
  CK(cudaGetLastError());
  if (ctx->d.cl_rec != (enable ? 1 : 0)) {  // the force kernel variant changes
    ctx->d.cl_rec = enable ? 1 : 0;
    CK(cudaStreamSynchronize(s));
    drop_graphs(ctx);
  }
  return CGDEM_OK;
}

int cgdem_get_closure_data(cgdem_ctx* ctx, float* out, int64_t rows, void* stream) {
  int r = ready(ctx);
  if (r) return r;
  if (!ctx->d.clblob) return fail(ctx, CGDEM_E_STATE, "the context was created without closure support");
  if (!out || rows < ctx->d.N) return fail(ctx, CGDEM_E_INVALID, "output must hold one row per particle");
  cudaStream_t s = st(stream);
  launch_closure_gather(ctx->d, s);
  if (ctx->d.N)
    CK(cudaMemcpyAsync(out, ctx->d.staging, sizeof(float) * CL_COLS * (size_t)ctx->d.N,
                       cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return check_status(ctx, s);
}

int cgdem_get_state(cgdem_ctx* ctx, double* x, double* v, double* w, double* F, double* T,
                    void* stream) {
  int r = ready(ctx);
  if (r) return r;
  cudaStream_t s = st(stream);
  const size_t N = ctx->d.N;
  launch_gather_state(ctx->d, s);
  double* outs[5] = {x, v, w, F, T};
  for (int k = 0; k < 5; ++k)
    if (outs[k] && N)
      CK(cudaMemcpyAsync(outs[k], ctx->d.staging + 3 * N * k, sizeof(double) * 3 * N,
                         cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return check_status(ctx, s);
}

int cgdem_get_contacts(cgdem_ctx* ctx, int32_t* id_i, int32_t* id_j, uint8_t* bonded, int64_t cap,
                       int64_t* count, void* stream) {
  int r = ready(ctx);
  if (r) return r;
  if (!count) return CGDEM_E_INVALID;
  cudaStream_t s = st(stream);
  Ctl c;
  CK(cudaMemcpyAsync(&c, ctx->d.ctl, sizeof c, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  uint32_t* buf = reinterpret_cast<uint32_t*>(ctx->d.rec[c.rec_cur ^ 1]);
  launch_collect_contacts(ctx->d, buf, ctx->contact_cap, s);
  unsigned long long n = 0;
  CK(cudaMemcpyAsync(&n, ctx->d.contact_n, sizeof n, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (n > ctx->contact_cap) return fail(ctx, CGDEM_E_CAPACITY, "too many contacts to collect");
  std::vector<uint32_t> h(2 * n);
  if (n) CK(cudaMemcpyAsync(h.data(), buf, sizeof(uint32_t) * 2 * n, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<uint64_t> key(n);
  for (size_t i = 0; i < n; ++i)
    key[i] = ((uint64_t)h[2 * i] << 32) | (uint64_t)h[2 * i + 1];
  std::sort(key.begin(), key.end(), [](uint64_t a, uint64_t b) {
    uint64_t ka = (a & 0xffffffff00000000ull) | (a & 0x7fffffffull);
    uint64_t kb = (b & 0xffffffff00000000ull) | (b & 0x7fffffffull);
    return ka < kb;
  });
  *count = (int64_t)n;
  const size_t m = std::min<size_t>(n, cap > 0 ? (size_t)cap : 0);
  for (size_t i = 0; i < m; ++i) {
    if (id_i) id_i[i] = (int32_t)(key[i] >> 32);
    if (id_j) id_j[i] = (int32_t)(key[i] & 0x7fffffffull);
    if (bonded) bonded[i] = (key[i] & 0x80000000ull) ? 1 : 0;
  }
  return check_status(ctx, s);
}

int cgdem_get_contact_springs(cgdem_ctx* ctx, int32_t* id_i, int32_t* id_j, double* xi, int64_t cap,
                              int64_t* count, void* stream) {
  int r = ready(ctx);
  if (r) return r;
  if (!count) return CGDEM_E_INVALID;
  cudaStream_t s = st(stream);
  Ctl c;
  CK(cudaMemcpyAsync(&c, ctx->d.ctl, sizeof c, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  // pairs (8 bytes) and springs (24 bytes) in the spare record buffer
  const size_t cap2 = ctx->contact_cap / 4;
  uint32_t* buf = reinterpret_cast<uint32_t*>(ctx->d.rec[c.rec_cur ^ 1]);
  double* xib = reinterpret_cast<double*>(buf + 2 * cap2);
  launch_collect_springs(ctx->d, buf, xib, cap2, s);
  unsigned long long n = 0;
  CK(cudaMemcpyAsync(&n, ctx->d.contact_n, sizeof n, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (n > cap2) return fail(ctx, CGDEM_E_CAPACITY, "too many contacts to collect");
  std::vector<uint32_t> h(2 * n);
  std::vector<double> hx(3 * n);
  if (n) {
    CK(cudaMemcpyAsync(h.data(), buf, sizeof(uint32_t) * 2 * n, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hx.data(), xib, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  std::vector<size_t> order(n);
  for (size_t i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](size_t a, size_t b) {
    if (h[2 * a] != h[2 * b]) return h[2 * a] < h[2 * b];
    return (h[2 * a + 1] & 0x7fffffffu) < (h[2 * b + 1] & 0x7fffffffu);
  });
  *count = (int64_t)n;
  const size_t m = std::min<size_t>(n, cap > 0 ? (size_t)cap : 0);
  for (size_t i = 0; i < m; ++i) {
    const size_t k = order[i];
    if (id_i) id_i[i] = (int32_t)h[2 * k];
    if (id_j) id_j[i] = (int32_t)(h[2 * k + 1] & 0x7fffffffu);
    if (xi)
      for (int c3 = 0; c3 < 3; ++c3) xi[3 * i + c3] = hx[3 * k + c3];
  }
  return check_status(ctx, s);
}

int cgdem_get_voidfrac(cgdem_ctx* ctx, uint64_t* cell_sums, int64_t cap, void* stream) {
  int r = ready(ctx);
  if (r) return r;
  if (!cell_sums || cap < ctx->d.Cf_total) return CGDEM_E_INVALID;
  cudaStream_t s = st(stream);
  Ctl c;
  CK(cudaMemcpyAsync(&c, ctx->d.ctl, sizeof c, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaMemcpyAsync(cell_sums, ctx->d.vf[c.vf_cur], sizeof(uint64_t) * ctx->d.Cf_total,
                     cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return check_status(ctx, s);
}

int cgdem_get_diagnostics(cgdem_ctx* ctx, double* out, int64_t cap, void* stream) {
  int r = ready(ctx);
  if (r) return r;
  if (!out || cap < 8 * ctx->d.n_samples) return CGDEM_E_INVALID;
  cudaStream_t s = st(stream);
  launch_diag(ctx->d, ctx->diag_part, s);
  CK(cudaMemcpyAsync(out, ctx->d.diag, sizeof(double) * 8 * ctx->d.n_samples,
                     cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return check_status(ctx, s);
}

int cgdem_get_fluid(cgdem_ctx* ctx, double* p, double* U, double* gradp, int64_t* reaction,
                    int64_t* iters, void* stream) {
  int r = ready(ctx);
  if (r) return r;
  cudaStream_t s = st(stream);
  const size_t nc = (size_t)ctx->d.Cf_total;
  if (!ctx->d.any_fluid) {
    if (p) std::fill(p, p + nc, 0.0);
    if (U) std::fill(U, U + 3 * nc, 0.0);
    if (gradp) std::fill(gradp, gradp + 3 * nc, 0.0);
    if (reaction) std::fill(reaction, reaction + 3 * nc, (int64_t)0);
    if (iters) *iters = 0;
    return CGDEM_OK;
  }
  Ctl c;
  CK(cudaMemcpyAsync(&c, ctx->d.ctl, sizeof c, cudaMemcpyDeviceToHost, s));
  std::vector<double4> u(nc), g(nc);
  if (p) CK(cudaMemcpyAsync(p, ctx->d.fl_p, sizeof(double) * nc, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(u.data(), ctx->d.Us, sizeof(double4) * nc, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(g.data(), ctx->d.gradp, sizeof(double4) * nc, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  // the last force evaluation's reaction buffer
  if (reaction)
    CK(cudaMemcpyAsync(reaction, ctx->d.react[c.step & 1], sizeof(int64_t) * 3 * nc, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<signed char> t(nc);
  CK(cudaMemcpy(t.data(), ctx->d.fl_type, nc, cudaMemcpyDeviceToHost));
  for (size_t k = 0; k < nc; ++k) {
    const double w = t[k] == 2 ? 0.0 : 1.0;  // cells of samples without Darcy flow hold zeros
    if (p && t[k] == 2) p[k] = 0.0;
    if (U) { U[3 * k] = w * u[k].x; U[3 * k + 1] = w * u[k].y; U[3 * k + 2] = w * u[k].z; }
    if (gradp) { gradp[3 * k] = w * g[k].x; gradp[3 * k + 1] = w * g[k].y; gradp[3 * k + 2] = w * g[k].z; }
  }
  if (iters) *iters = c.fl_iters;
  return check_status(ctx, s);
}

int cgdem_bond_touching(cgdem_ctx* ctx, void* stream) {
  int r = ready(ctx);
  if (r) return r;
  launch_bond_touching(ctx->d, st(stream));
  CK(cudaGetLastError());
  return CGDEM_OK;
}

int cgdem_set_stage(cgdem_ctx* ctx, int sample, const cgdem_stage* stg, void* stream) {
  int r = ready(ctx);
  if (r) return r;
  if (!stg || sample < 0 || sample >= (int)ctx->sd.size()) return fail(ctx, CGDEM_E_INVALID, "bad sample or stage");
  const cgdem_sample_params& p = ctx->sp[sample];
  SampleDev& S = ctx->sd[sample];
  if (stg->jkr_mode != 0 && stg->jkr_mode != 1) return fail(ctx, CGDEM_E_INVALID, "jkr_mode must be 0 or 1");
  if (ctx->d.clblob) return fail(ctx, CGDEM_E_INVALID, "preparation stages run in contexts without the learned closure");
  if (!(2.0 * jkr_reach(S.gamma, S.Es, 0.5 * p.r_max, stg->jkr_mode) < p.skin))
    return fail(ctx, CGDEM_E_INVALID, "skin %.3g must exceed twice the separation of the contact model",
                p.skin);
  if ((stg->plate_mode != 0 || stg->pen_mode != 0) && S.kind != CGDEM_CYLINDER)
    return fail(ctx, CGDEM_E_INVALID, "moving boundaries need a cylinder sample");
  if ((stg->plate_mode != 0 && stg->plate_mode != 1) || stg->pen_mode < 0 || stg->pen_mode > 2)
    return fail(ctx, CGDEM_E_INVALID, "plate_mode must be 0 or 1, pen_mode 0, 1 or 2");
  if (stg->plate_H > S.H) return fail(ctx, CGDEM_E_INVALID, "plate_H above the sample's H");
  if (stg->plate_mode == 1 && !(stg->plate_gain > 0 && stg->plate_vmax > 0 && std::isfinite(stg->plate_stress)))
    return fail(ctx, CGDEM_E_INVALID, "a moving plate needs plate_gain > 0, plate_vmax > 0, a finite stress");
  if (stg->pen_mode != 0 && !(stg->pen_radius > 0 && stg->pen_speed > 0 && stg->pen_z_stop < stg->pen_z_start &&
                              stg->pen_force >= 0))
    return fail(ctx, CGDEM_E_INVALID, "a penetrometer needs pen_radius > 0, pen_speed > 0, pen_z_stop < pen_z_start");
  cudaStream_t s = st(stream);
  StageDev W;
  CK(cudaMemcpyAsync(&W, ctx->d.stage + sample, sizeof W, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  W.plate_mode = stg->plate_mode;
  W.plate_stress = stg->plate_stress;
  W.plate_gain = stg->plate_gain;
  W.plate_vmax = stg->plate_vmax;
  if (stg->plate_H > 0) W.H = stg->plate_H;
  if (stg->plate_mode != 1) W.v_plate = 0.0;
  if (stg->pen_mode == 2 && W.pen_dir == 0) return fail(ctx, CGDEM_E_INVALID, "no penetrometer to pull back");
  W.pen_radius = stg->pen_radius;
  W.pen_speed = stg->pen_speed;
  W.pen_z_start = stg->pen_z_start;
  W.pen_z_stop = stg->pen_z_stop;
  W.pen_force = stg->pen_force;
  if (stg->pen_mode == 2) {  // the tool goes back up from where it is
    W.pen_dir = 1;
    W.v_pen = stg->pen_speed;
  } else {
    W.pen_z = stg->pen_z_start;
    W.pen_dir = stg->pen_mode == 1 ? -1 : 0;
    W.v_pen = stg->pen_mode == 1 ? -stg->pen_speed : 0.0;
  }
  W.outlet_closed = stg->outlet_closed ? 1 : 0;
  CK(cudaMemcpyAsync(ctx->d.stage + sample, &W, sizeof W, cudaMemcpyHostToDevice, s));
  S.jkr_mode = stg->jkr_mode;
  ctx->sp[sample].jkr_mode = stg->jkr_mode;
  CK(cudaMemcpyAsync(&ctx->d.sp[sample].jkr_mode, &S.jkr_mode, sizeof(int), cudaMemcpyHostToDevice, s));
  // a new penetrometer starts without spring history
  if (S.kind == CGDEM_CYLINDER && stg->pen_mode != 2) launch_clear_wall_history(ctx->d, sample, 3, s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  if (!ctx->d.prep) {  // from now on the force kernels that run the stages (graphs recaptured)
    ctx->d.prep = 1;
    drop_graphs(ctx);
  }
  return CGDEM_OK;
}

int cgdem_get_boundaries(cgdem_ctx* ctx, double* out, int64_t cap, void* stream) {
  int r = ready(ctx);
  if (r) return r;
  const int S = (int)ctx->sd.size();
  if (!out || cap < 6 * (int64_t)S) return fail(ctx, CGDEM_E_INVALID, "out needs 6 doubles per sample");
  cudaStream_t s = st(stream);
  std::vector<StageDev> W(S);
  CK(cudaMemcpyAsync(W.data(), ctx->d.stage, sizeof(StageDev) * S, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int k = 0; k < S; ++k) {
    const double Rc = ctx->sd[k].Rc;
    out[6 * k + 0] = W[k].H;
    out[6 * k + 1] = W[k].v_plate;
    out[6 * k + 2] = ctx->sd[k].kind == CGDEM_CYLINDER
                         ? (double)W[k].plate_q_last * 9.094947017729282379150390625e-13 / (PI * Rc * Rc)
                         : 0.0;
    out[6 * k + 3] = W[k].pen_z;
    out[6 * k + 4] = (double)W[k].pen_dir;
    out[6 * k + 5] = (double)W[k].pen_q_last * 9.094947017729282379150390625e-13;
  }
  return CGDEM_OK;
}

int cgdem_set_psd_classes(cgdem_ctx* ctx, const double* edges, int nclass, void* stream) {
  if (!ctx) return CGDEM_E_INVALID;
  if (nclass < 0 || nclass > CGDEM_PSD_MAX || (nclass > 0 && !edges))
    return fail(ctx, CGDEM_E_INVALID, "nclass must lie in [0, %d] with nclass + 1 edges", CGDEM_PSD_MAX);
  for (int c = 0; c < nclass; ++c)
    if (!(edges[c] < edges[c + 1]) || !(edges[c] >= 0.0))
      return fail(ctx, CGDEM_E_INVALID, "class edges must be non-negative and increasing");
  for (auto& S : ctx->sd) {
    S.n_psd = nclass;
    for (int c = 0; c <= CGDEM_PSD_MAX; ++c) S.psd_edge[c] = c <= nclass && nclass ? edges[c] : 0.0;
  }
  cudaStream_t s = st(stream);
  CK(cudaMemcpyAsync(ctx->d.sp, ctx->sd.data(), sizeof(SampleDev) * ctx->sd.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(ctx->d.psd_count, 0, sizeof(unsigned long long) * CGDEM_PSD_MAX * ctx->d.n_samples, s));
  CK(cudaMemsetAsync(ctx->d.psd_mass, 0, sizeof(unsigned long long) * CGDEM_PSD_MAX * ctx->d.n_samples, s));
  CK(cudaStreamSynchronize(s));
  return CGDEM_OK;
}

int cgdem_get_produced_psd(cgdem_ctx* ctx, double* mass, int64_t* count, int64_t cap, void* stream) {
  int r = ready(ctx);
  if (r) return r;
  const int S = ctx->d.n_samples;
  if (cap < (int64_t)CGDEM_PSD_MAX * S) return fail(ctx, CGDEM_E_INVALID, "output needs %d entries per sample",
                                                     CGDEM_PSD_MAX);
  cudaStream_t s = st(stream);
  std::vector<unsigned long long> c((size_t)CGDEM_PSD_MAX * S), q((size_t)CGDEM_PSD_MAX * S);
  CK(cudaMemcpyAsync(c.data(), ctx->d.psd_count, sizeof(unsigned long long) * c.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(q.data(), ctx->d.psd_mass, sizeof(unsigned long long) * q.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int k = 0; k < S; ++k)
    for (int j = 0; j < CGDEM_PSD_MAX; ++j) {
      const size_t i = (size_t)k * CGDEM_PSD_MAX + j;
      if (count) count[i] = (int64_t)c[i];
      if (mass) mass[i] = (double)q[i] * ctx->sd[k].psd_mq;
    }
  return check_status(ctx, s);
}

int cgdem_get_removed_step(cgdem_ctx* ctx, int32_t* removed_step, void* stream) {
  int r = ready(ctx);
  if (r) return r;
  if (!removed_step) return CGDEM_E_INVALID;
  cudaStream_t s = st(stream);
  if (ctx->d.N)
    CK(cudaMemcpyAsync(removed_step, ctx->d.removed_step, sizeof(int) * ctx->d.N,
                       cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return check_status(ctx, s);
}

int cgdem_get_counters(cgdem_ctx* ctx, int64_t* steps, int64_t* rebuilds, int32_t* max_candidates,
                       int64_t* total_candidates, void* stream) {
  int r = ready(ctx);
  if (r) return r;
  cudaStream_t s = st(stream);
  Ctl c;
  CK(cudaMemcpyAsync(&c, ctx->d.ctl, sizeof c, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (steps) *steps = c.step;
  if (rebuilds) *rebuilds = c.rebuilds;
  if (max_candidates) *max_candidates = c.max_cand;
  if (total_candidates) *total_candidates = c.cand_total;
  return CGDEM_OK;
}

int cgdem_get_launch_counts(cgdem_ctx* ctx, int64_t* step_kernels, int32_t* rebuild_kernels) {
  if (!ctx) return CGDEM_E_INVALID;
  if (step_kernels) *step_kernels = ctx->step_kernels;
  if (rebuild_kernels) *rebuild_kernels = ctx->rebuild_kernels;
  return CGDEM_OK;
}

int cgdem_profile_step(cgdem_ctx* ctx, int64_t nsteps, double* out, void* stream) {
  int r = ready(ctx);
  if (r) return r;
  if (!out || nsteps < 2) return fail(ctx, CGDEM_E_INVALID, "profile needs nsteps >= 2 and out");
  cudaStream_t s = st(stream);
  Ctl c0;
  CK(cudaMemcpyAsync(&c0, ctx->d.ctl, sizeof c0, cudaMemcpyDeviceToHost, s));
  const int64_t body = nsteps - 1;
  std::vector<cudaEvent_t> ev(3 * body + 2);
  for (auto& e : ev) CK(cudaEventCreate(&e));
  CK(cudaEventRecord(ev[0], s));
  launch_kick_drift(ctx->d, 1, s);
  for (int64_t i = 0; i < body; ++i) {
    CK(cudaEventRecord(ev[1 + 3 * i], s));
    launch_rebuild(ctx->d, s);
    CK(cudaEventRecord(ev[2 + 3 * i], s));
    launch_forces(ctx->d, 1, ctx->cfg.block_size, s, 0);
    CK(cudaEventRecord(ev[3 + 3 * i], s));
    if (ctx->any_cube) launch_cube_after_mid(ctx->d, s);
  }
  launch_rebuild(ctx->d, s);
  launch_forces(ctx->d, 2, ctx->cfg.block_size, s, 0);
  CK(cudaEventRecord(ev[3 * body + 1], s));
  CK(cudaStreamSynchronize(s));
  double force = 0, rebuild = 0, floor_ms = 1e30;
  for (int64_t i = 0; i < body; ++i) {
    float a = 0, b = 0;
    CK(cudaEventElapsedTime(&a, ev[1 + 3 * i], ev[2 + 3 * i]));
    CK(cudaEventElapsedTime(&b, ev[2 + 3 * i], ev[3 + 3 * i]));
    rebuild += a;
    force += b;
    floor_ms = std::min(floor_ms, (double)a);
  }
  rebuild -= floor_ms * (double)body;
  float tot = 0;
  CK(cudaEventElapsedTime(&tot, ev[0], ev[3 * body + 1]));
  for (auto& e : ev) cudaEventDestroy(e);
  Ctl c1;
  CK(cudaMemcpy(&c1, ctx->d.ctl, sizeof c1, cudaMemcpyDeviceToHost));
  out[0] = force / (double)body;
  out[1] = rebuild;
  out[2] = (double)(c1.rebuilds - c0.rebuilds);
  out[3] = tot;
  out[4] = (double)body;
  out[5] = floor_ms;
  return check_status(ctx, s);
}

}  // extern "C"
