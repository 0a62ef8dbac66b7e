// k_forces.cu -- contact, wall, body and drag forces of one DEM step fused
// with the velocity-Verlet update (arXiv 2211.06142, Sec. 2.1-2.3).
//
// Two kernels, one per precision, share the per-sphere end of the step
// (finish_step: walls, gravity, buoyancy, drag, integration, porosity
// scatter, closure network, bookkeeping).  Every sum runs in a fixed order,
// so the step is deterministic and needs no floating-point atomics.
//
// Mixed precision (k_forces_lanes) -- positions, integrator and accumulators
// stay FP64; the contact geometry comes from a 32-bit fixed-point shadow of
// the positions (exact integer differences, so delta = Ri + Rj - d suffers no
// cancellation); contact physics and tangential history run in FP32.  Every
// integer decision (touching, bond break) is taken in IEEE double from the
// FP64 positions whenever the fixed-point value lies within its error band of
// the threshold, so it always equals the FP64 decision.  Every pair is listed
// from both sides and evaluated twice (bit-identical magnitudes); one lane
// walks one sphere's list.  The rebuild stores the spheres of each tile of
// 1024 (in cell order) by decreasing list length, so a warp's lanes have
// lists of about the same length, and lays the records out entry-major per
// warp, so each step of the walk reads one contiguous line.  The kernel is
// bound by latency (dependent chains of the contact law, the partner
// gathers), not by arithmetic or bandwidth.
//
// FP64 (k_forces_pairs) -- geometry and contact physics in double.  GB300
// runs FP64 at two operations per SM per clock, so each pair is listed once,
// by its lower-index sphere (the owner): the owner's warp writes the pair's
// result (the force on the owner and n x F_t) into the partner's inbox slot,
// publishes that its segment is done, waits until the segments owning its
// spheres' lower-index partners have published (blocks take segments in the
// order they start, from a counter, so every warp waited on is running and
// publishes before it waits itself) and adds its inbox in slot order.
#include "cgdem_internal.cuh"
#include "tc05.cuh"

namespace cgdem {

constexpr double PI_D = 3.14159265358979323846;
constexpr float PI_F = 3.14159265358979323846f;
#ifndef CGDEM_FORCE_MINB
#define CGDEM_FORCE_MINB 3  // resident 256-thread blocks per SM the register budget must allow
#endif
#ifndef CGDEM_PAIRS_MINB
// the same for the FP64 kernel: it is bound by the FP64 pipe, and 128
// registers a thread (two blocks) ran faster than 80 (three): 0.570 against
// 0.610 ms on the 200k cylinder, 4.23 against 4.27 ms at 1.97M spheres
#define CGDEM_PAIRS_MINB 2
#endif
constexpr int FORCE_BLOCK_MAX = 256;  // launches use 64, 128 or 256 threads (autotuned)
constexpr unsigned FULL = 0xffffffffu;

template <typename T>
struct Consts;
template <>
struct Consts<float> {
  static __device__ __forceinline__ float damp() { return 1.8257418583505538f; }  // 2 sqrt(5/6)
  static __device__ __forceinline__ float pi() { return PI_F; }
  static constexpr int newton_iters = 4;
};
template <>
struct Consts<double> {
  static __device__ __forceinline__ double damp() { return 1.8257418583505538; }
  static __device__ __forceinline__ double pi() { return PI_D; }
  static constexpr int newton_iters = 5;  // from within ~5 % of the root: 1 ulp after 5 steps
};

// Elementary functions of the contact law.  Double: correctly rounded or
// within a few 1e-16 (the FP64 tolerance against the oracle is 1e-10).  Float
// (the mixed mode, toleranced at 1e-4 against the FP64 oracle and with every
// integer decision taken in FP64): hardware approximations of a few ulp --
// reciprocal square root, base-2 logarithm and exponential, fast divide --
// which cost one to three instructions instead of an IEEE sequence.
__device__ __forceinline__ double m_sqrt(double a) { return sqrt(a); }
__device__ __forceinline__ double m_div(double a, double b) { return a / b; }
__device__ __forceinline__ double m_cbrt(double a) { return cbrt(a); }
__device__ __forceinline__ double m_exp(double a) { return exp(a); }
__device__ __forceinline__ double m_log10(double a) { return log10(a); }
// a^b for a > 0 as 2^(b log2 a): the exponent's rounding error (|b log2 a| < 10
// here) moves the result by a few 1e-16 relative, and the general pow's
// extra-precision path costs several times more FP64 work
__device__ __forceinline__ double m_pow(double a, double b) { return exp2(b * log2(a)); }
__device__ __forceinline__ float m_sqrt(float a) { return a > 0.f ? a * rsqrtf(a) : 0.f; }
__device__ __forceinline__ float m_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ float m_cbrt(float a) {
  return a > 0.f ? exp2f(__log2f(a) * (1.0f / 3.0f)) : 0.f;
}
__device__ __forceinline__ float m_exp(float a) { return __expf(a); }
__device__ __forceinline__ float m_log10(float a) { return __log10f(a); }
__device__ __forceinline__ float m_pow(float a, float b) { return exp2f(b * __log2f(a)); }

// Contact radius and elastic normal force on the stable JKR branch
// (Eq. 12-13), solved in reduced units: with a_A^3 = 4 pi gamma R*^2 / E*
// (Table 1, point A) and u^2 = a / a_A, Eq. 13 reads u^4 - u = delta / d_A
// with d_A = a_A^2 / R*, and Eq. 12 reads F = pi gamma R* (16/3 u^6 - 8 u^3).
// Newton from above converges monotonically (the quartic is convex and
// increasing for u > u_S = 4^(-1/3), point S; the modified JKR's branch
// starts at u_C = (3/4)^(1/3), point C).  The original JKR (orig) also runs
// between S and C, D_S <= D < D_C: there Newton starts from u_S + t with
// 6 u_S^2 t^2 = D - D_S, the root of the quartic's expansion at S to second
// order, which lies above the root (the cubic and quartic terms are positive).
template <typename T>
__device__ __forceinline__ T jkr_start(T D, bool orig) {
  const T uS = T(0.6299605249474366), DS = T(-0.4724703937105774), DC = T(-0.22714007410401746);
  if (orig && D < DC) {
    const T t2 = m_div(D - DS, T(2.381101577952299));  // (D - D_S) / (6 u_S^2)
    return uS + (t2 > T(0) ? m_sqrt(t2) : T(0));
  }
  return D >= T(0) ? m_sqrt(m_sqrt(D + T(1))) + T(0.05) : T(1);
}

template <typename T>
__device__ __forceinline__ void jkr_solve(T delta, T Rs, T Es, T gamma, bool orig, T* a_out, T* F_out) {
  const T pi = Consts<T>::pi();
  T aA = m_cbrt(m_div(T(4) * pi * gamma * Rs * Rs, Es));
  T dA = m_div(aA * aA, Rs);
  T D = m_div(delta, dA);
  T u = jkr_start<T>(D, orig);
#pragma unroll
  for (int it = 0; it < Consts<T>::newton_iters; ++it) {
    T u3 = u * u * u;
    u -= m_div(u3 * u - u - D, T(4) * u3 - T(1));
  }
  const T uLo = orig ? T(0.6299605249474366) : T(0.90856029641606983);  // u_S or u_C
  if (u < uLo) u = uLo;
  T u3 = u * u * u;
  *a_out = u * u * aA;
  *F_out = pi * gamma * Rs * (T(16) / T(3) * u3 * u3 - T(8) * u3);
}

// The contact law shared by pairs and walls (Eq. 4, 5, 12, 13, 32-35).
// n: unit normal from i to the partner; vrel: partner velocity minus own;
// vc: relative surface velocity at the contact.  Returns the force on i.
template <typename T>
__device__ __forceinline__ void contact_law(T delta, V3<T> n, V3<T> vrel, V3<T> vc, T Rs, T ms,
                                            T gamma, bool bonded, T Es, T Gs, T beta, T mu, T dt,
                                            int coulomb_mode, V3<T>& xi, V3<T>& Fi, V3<T>& Ft,
                                            bool orig = false) {
  T a, Fne;
  if (bonded && gamma > T(0)) {
    jkr_solve<T>(delta, Rs, Es, gamma, orig, &a, &Fne);
  } else {
    a = delta > T(0) ? m_sqrt(Rs * delta) : T(0);
    Fne = m_div(T(4) * Es * a * a * a, T(3) * Rs);
  }
  const T cd = Consts<T>::damp();
  T gn = cd * beta * m_sqrt(T(2) * Es * a * ms);  // Eq. 32
  T vn = dot3(vrel, n);
  T Fn = Fne - gn * vn;
  // tangential spring rotated into the tangent plane, Eq. 4
  T vcn = dot3(vc, n);
  V3<T> vt = v3<T>(vc.x - vcn * n.x, vc.y - vcn * n.y, vc.z - vcn * n.z);
  T old = m_sqrt(dot3(xi, xi));
  T xn = dot3(xi, n);
  xi.x -= xn * n.x;
  xi.y -= xn * n.y;
  xi.z -= xn * n.z;
  T nw = m_sqrt(dot3(xi, xi));
  if (nw > T(0)) {
    T sc = m_div(old, nw);
    xi.x *= sc;
    xi.y *= sc;
    xi.z *= sc;
  } else {
    xi = v3<T>(0, 0, 0);
  }
  xi.x += vt.x * dt;
  xi.y += vt.y * dt;
  xi.z += vt.z * dt;
  T kt = T(8) * Gs * a;
  T gt = cd * beta * m_sqrt(kt * ms);
  Ft = v3<T>(kt * xi.x + gt * vt.x, kt * xi.y + gt * vt.y, kt * xi.z + gt * vt.z);
  T FC = T(3) * Consts<T>::pi() * gamma * Rs;  // Table 1
  T Flim = coulomb_mode == 1 ? fabs(Fne) : (bonded ? Fne + T(2) * FC : Fne);
  if (Flim < T(0)) Flim = T(0);
  T ftm = m_sqrt(dot3(Ft, Ft));
  T cap = mu * Flim;  // Eq. 35
  if (ftm > cap) {
    T sc = ftm > T(0) ? m_div(cap, ftm) : T(0);
    Ft.x *= sc;
    Ft.y *= sc;
    Ft.z *= sc;
    if (kt > T(0)) {
      const T ik = m_div(T(1), kt);
      xi.x = (Ft.x - gt * vt.x) * ik;
      xi.y = (Ft.y - gt * vt.y) * ik;
      xi.z = (Ft.z - gt * vt.z) * ik;
    }
  }
  Fi = v3<T>(-Fn * n.x + Ft.x, -Fn * n.y + Ft.y, -Fn * n.z + Ft.z);
}

// The contact law of the mixed step in FP32: the terms of contact_law in an
// order that shares work between them.  Bonded pairs (stable JKR branch,
// Eq. 12-13) take d_A = a_A^2 / R* = 16^(1/3) (pi^2 gamma^2 R* / E*^2)^(1/3),
// which the caller has for the bond-break test, and start Newton's method on
// u^4 - u = delta / d_A from (delta / d_A + 1)^(1/4) (exact at delta = 0,
// within 4 % on the branch): three steps reach 2e-10 relative.  Unbonded
// pairs: Hertz with a^2 = R* delta, so 4 E* a^3 / (3 R*) = (4/3) E* a delta.
// Damping (Eq. 32) and the tangential dashpot share sqrt(a m*); the spring
// keeps its length through one square root and one reciprocal square root;
// the Coulomb test (Eq. 35) compares squares and takes the root only when the
// spring slips.
__device__ __forceinline__ void contact_law_mixed(float delta, V3<float> n, V3<float> vrel, V3<float> vc,
                                                  float Rs, float ms, float gamma, bool bonded, float dA,
                                                  const SampleDev& S, V3<float>& xi, V3<float>& Fi,
                                                  V3<float>& Ft, bool orig) {
  float a, Fne;
  if (bonded && gamma > 0.f) {
    const float D = __fdividef(delta, dA);
    float u = (orig && D < -0.22714007410401746f) ? jkr_start<float>(D, true) : m_sqrt(m_sqrt(D + 1.f));
#pragma unroll
    for (int it = 0; it < 3; ++it) {
      const float u3 = u * u * u;
      u -= __fdividef(u3 * u - u - D, 4.f * u3 - 1.f);
    }
    const float uLo = orig ? 0.6299605249474366f : 0.90856029641606983f;  // u_S or u_C
    if (u < uLo) u = uLo;
    const float u3 = u * u * u;
    a = u * u * m_sqrt(dA * Rs);
    Fne = PI_F * gamma * Rs * (16.f / 3.f * u3 * u3 - 8.f * u3);
  } else {
    a = delta > 0.f ? m_sqrt(Rs * delta) : 0.f;
    Fne = (4.f / 3.f) * S.Es_f * a * delta;
  }
  const float sq = m_sqrt(a * ms);
  const float vn = dot3(vrel, n);
  const float Fn = Fne - S.cdbn_f * sq * vn;  // Eq. 32
  // tangential spring rotated into the tangent plane, Eq. 4
  const float vcn = dot3(vc, n);
  const V3<float> vt = v3<float>(vc.x - vcn * n.x, vc.y - vcn * n.y, vc.z - vcn * n.z);
  const float old2 = dot3(xi, xi);
  const float xn = dot3(xi, n);
  xi.x -= xn * n.x;
  xi.y -= xn * n.y;
  xi.z -= xn * n.z;
  const float nw2 = dot3(xi, xi);
  if (nw2 > 0.f) {
    const float sc = m_sqrt(old2) * rsqrtf(nw2);
    xi.x *= sc;
    xi.y *= sc;
    xi.z *= sc;
  } else {
    xi = v3<float>(0, 0, 0);
  }
  const float dt = S.dt_f;
  xi.x += vt.x * dt;
  xi.y += vt.y * dt;
  xi.z += vt.z * dt;
  const float kt = 8.f * S.Gs_f * a;
  const float gt = S.cdbt_f * sq;
  Ft = v3<float>(kt * xi.x + gt * vt.x, kt * xi.y + gt * vt.y, kt * xi.z + gt * vt.z);
  const float FC = 3.f * PI_F * gamma * Rs;  // Table 1
  float Flim = S.coulomb_mode == 1 ? fabsf(Fne) : (bonded ? Fne + 2.f * FC : Fne);
  if (Flim < 0.f) Flim = 0.f;
  const float cap = S.mu_f32 * Flim;  // Eq. 35
  const float ft2 = dot3(Ft, Ft);
  if (ft2 > cap * cap) {
    const float sc = cap * rsqrtf(ft2);
    Ft.x *= sc;
    Ft.y *= sc;
    Ft.z *= sc;
    if (kt > 0.f) {
      const float ik = __fdividef(1.f, kt);
      xi.x = (Ft.x - gt * vt.x) * ik;
      xi.y = (Ft.y - gt * vt.y) * ik;
      xi.z = (Ft.z - gt * vt.z) * ik;
    }
  }
  Fi = v3<float>(-Fn * n.x + Ft.x, -Fn * n.y + Ft.y, -Fn * n.z + Ft.z);
}

// Reciprocal and cube root in FP64 by Newton-Raphson iteration from an FP32
// seed, in place of the IEEE divide and the library cube root, for results
// that feed forces only (never an integer decision): the iteration converges
// quadratically, so a seed good to about 2^-21 is good to about 2^-42 after
// one step and to the rounding of the last step after two (within about one
// ulp of the correctly rounded value).  The cube root's step uses the FP32
// reciprocal of its derivative 3 x^2; the error that leaves in each step is
// the derivative's (2^-21) times the step's own, so two steps still reach the
// last bit.  Outside 2^-100 <= |x| < 2^101, where a seed could leave the
// FP32 normal range, they fall back to the IEEE operation.
//
// The seeds move between FP64 and FP32 by integer operations on the bits
// (seed_f truncates the mantissa; widen_f is exact for a normal float), and
// tests of a double's sign, or the order of two non-negative doubles, compare
// bit patterns as integers (exact): the FP64 step is bound by the FP64 pipe,
// which runs conversions and floating-point compares as well as arithmetic.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ bool seed_range(double x) {
  const unsigned e = ((unsigned)__double2hiint(x) >> 20) & 0x7ffu;
  return e - 923u <= 200u;
}
__device__ __forceinline__ float seed_f(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = ((hi >> 20) & 0x7ffu) - 896u;
  return __uint_as_float((hi & 0x80000000u) | (e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}
__device__ __forceinline__ double widen_f(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned hi = (u & 0x80000000u) | ((((u >> 23) & 0xffu) + 896u) << 20) | ((u & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
}

__device__ __forceinline__ double nr_rcp(double b) {
  if (!seed_range(b)) return 1.0 / b;
  double r = widen_f(__fdividef(1.0f, seed_f(b)));
  double e = fma(-b, r, 1.0);
  r = fma(r, e, r);
  e = fma(-b, r, 1.0);
  return fma(r, e, r);
}

__device__ __forceinline__ double nr_cbrt(double v) {
  if (!seed_range(v) || dbits(v) < 0) return cbrt(v);
  double x = widen_f(m_cbrt(seed_f(v)));
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const float xf = seed_f(x);
    const double r = widen_f(__fdividef(1.0f, 3.0f * xf * xf));
    x = fma(-fma(x * x, x, -v), r, x);
  }
  return x;
}

// nr_rcp and nr_cbrt beside CUDA's 1 / x and cbrt(|x|) on n inputs:
// out[4 i .. 4 i + 3] = nr_rcp(x), 1 / x, nr_cbrt(|x|), cbrt(|x|).
__global__ void k_fp64_math_check(const double* x, int64_t n, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i], a = fabs(v);
    out[4 * i] = nr_rcp(v);
    out[4 * i + 1] = 1.0 / v;
    out[4 * i + 2] = a > 0.0 ? nr_cbrt(a) : 0.0;
    out[4 * i + 3] = cbrt(a);
  }
}

void launch_fp64_math_check(const double* x, int64_t n, double* out, cudaStream_t s) {
  if (n > 0) k_fp64_math_check<<<152 * 4, 256, 0, s>>>(x, n, out);
}

// The contact law of the FP64 step for the modified JKR and Hertz: the
// terms of contact_law with the work shared as in the mixed law, in FP64.
// The stable JKR branch (Eq. 12-13): a_A^3 = 4 pi gamma R*^2 / E* by nr_cbrt,
// D = delta R* / a_A^2; u^4 - u = D is solved first in FP32 (three Newton
// steps from (D + 1)^(1/4), to about 1e-7), then by two FP64 Newton steps
// whose derivative reciprocal is taken in FP32 (the error left per step is
// the reciprocal's 2^-21 times the step's own: 1e-7 -> 1e-13 -> 1e-19, and
// 4 u^3 - 1 >= 2 on the branch, u >= u_C).  Damping (Eq. 32) and the
// tangential dashpot share sqrt(a m*); the spring keeps its length with one
// square root; the Coulomb test (Eq. 35) compares squares.
__device__ __forceinline__ void contact_law_fp64(double delta, V3<double> n, V3<double> vrel, V3<double> vc,
                                                 double Rs, double ms, double gamma, bool bonded,
                                                 const SampleDev& S, V3<double>& xi, V3<double>& Fi,
                                                 V3<double>& Ft) {
  double a, Fne;
  if (bonded && dbits(gamma) > 0) {
    const double aA = nr_cbrt(4.0 * PI_D * gamma * Rs * Rs * S.inv_Es);
    const double D = delta * Rs * nr_rcp(aA * aA);
    const float Df = seed_range(D) ? seed_f(D) : __double2float_rn(D);
    float uf = m_sqrt(m_sqrt(Df + 1.f));
#pragma unroll
    for (int it = 0; it < 3; ++it) {
      const float u3 = uf * uf * uf;
      uf -= __fdividef(u3 * uf - uf - Df, 4.f * u3 - 1.f);
    }
    double u = widen_f(uf);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      const double u3 = u * u * u;
      const double r = widen_f(__fdividef(1.0f, 4.f * seed_f(u3) - 1.f));
      u = fma(-(fma(u3, u, -u) - D), r, u);
    }
    const double uC = 0.90856029641606983;  // u_C
    if (dbits(u) < dbits(uC)) u = uC;
    const double u3 = u * u * u;
    a = u * u * aA;
    Fne = PI_D * gamma * Rs * (16.0 / 3.0 * u3 * u3 - 8.0 * u3);
  } else {
    a = dbits(delta) > 0 ? sqrt(Rs * delta) : 0.0;
    Fne = (4.0 / 3.0) * S.Es * a * delta;
  }
  const double sq = sqrt(a * ms);
  const double vn = dot3(vrel, n);
  const double Fn = Fne - S.cdbn * sq * vn;  // Eq. 32
  // tangential spring rotated into the tangent plane, Eq. 4
  const double vcn = dot3(vc, n);
  const V3<double> vt = v3<double>(vc.x - vcn * n.x, vc.y - vcn * n.y, vc.z - vcn * n.z);
  const double old2 = dot3(xi, xi);
  const double xn = dot3(xi, n);
  xi.x -= xn * n.x;
  xi.y -= xn * n.y;
  xi.z -= xn * n.z;
  const double nw2 = dot3(xi, xi);
  if (dbits(nw2) > 0) {
    const double sc = sqrt(old2 * nr_rcp(nw2));
    xi.x *= sc;
    xi.y *= sc;
    xi.z *= sc;
  } else {
    xi = v3<double>(0, 0, 0);
  }
  const double dt = S.dt;
  xi.x += vt.x * dt;
  xi.y += vt.y * dt;
  xi.z += vt.z * dt;
  const double kt = 8.0 * S.Gs * a;
  const double gt = S.cdbt * sq;
  Ft = v3<double>(kt * xi.x + gt * vt.x, kt * xi.y + gt * vt.y, kt * xi.z + gt * vt.z);
  const double FC = 3.0 * PI_D * gamma * Rs;  // Table 1
  double Flim = S.coulomb_mode == 1 ? fabs(Fne) : (bonded ? Fne + 2.0 * FC : Fne);
  if (dbits(Flim) < 0) Flim = 0.0;
  const double cap = S.mu * Flim;  // Eq. 35
  const double ft2 = dot3(Ft, Ft);
  if (dbits(ft2) > dbits(cap * cap)) {
    const double sc = cap * nr_rcp(sqrt(ft2));
    Ft.x *= sc;
    Ft.y *= sc;
    Ft.z *= sc;
    if (dbits(kt) > 0) {
      const double ik = nr_rcp(kt);
      xi.x = (Ft.x - gt * vt.x) * ik;
      xi.y = (Ft.y - gt * vt.y) * ik;
      xi.z = (Ft.z - gt * vt.z) * ik;
    }
  }
  Fi = v3<double>(-Fn * n.x + Ft.x, -Fn * n.y + Ft.y, -Fn * n.z + Ft.z);
}

// Di Felice drag (Eq. 8-11) written as (pi d^2 / 8) (0.63 sqrt(rho_f |w|)
// + 4.8 sqrt(mu_f / d))^2 w n^-chi, which equals Eq. 8 with Eq. 9 and stays
// finite as Re -> 0.
template <typename T>
__device__ __forceinline__ V3<T> drag_force(T rho_f, T mu_f, T dp, V3<T> w, T n) {
  T wm = m_sqrt(dot3(w, w));
  if (!(wm > T(0))) return v3<T>(0, 0, 0);
  T Re = m_div(rho_f * dp * wm, mu_f);
  T lr = T(1.5) - m_log10(Re);
  T chi = T(3.7) - T(0.65) * m_exp(-(lr * lr) * T(0.5));
  T t = T(0.63) * m_sqrt(rho_f * wm) + T(4.8) * m_sqrt(m_div(mu_f, dp));
  T pre = Consts<T>::pi() * dp * dp * T(0.125) * t * t * m_pow(n, -chi);
  return v3<T>(pre * w.x, pre * w.y, pre * w.z);
}

enum { MODE_FORCES = 0, MODE_MID = 1, MODE_CANON = 2 };

// Flags and data that other blocks of the same launch write: the flag with
// acquire / release semantics at GPU scope, the data from L2 (not L1).
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* a) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* a, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}
__device__ __forceinline__ double4 ldcg_d4(const double4* a) {
  const double2* b = reinterpret_cast<const double2*>(a);
  const double2 u = __ldcg(b), w = __ldcg(b + 1);
  return make_double4(u.x, u.y, w.x, w.y);
}
constexpr int WAIT_LIMIT = 1 << 22;  // polls of a segment flag before the step reports a timeout

// Bring a line into L1 ahead of use (no register is held meanwhile).
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// 64-bit integers to float through 32-bit halves (both non-negative, so the
// sum has no cancellation): relative error below 2^-23, no 64-bit conversion.
__device__ __forceinline__ float u64_to_f(unsigned long long v) {
  return fmaf((float)(unsigned)(v >> 32), 4294967296.0f, (float)(unsigned)v);
}
__device__ __forceinline__ float s64_to_f(long long v) {
  const float m = u64_to_f((unsigned long long)(v < 0 ? -v : v));
  return v < 0 ? -m : m;
}

// Penetrometer contact (Sec. 3.1): the tool is a solid cylinder of radius
// rp on the axis with a hemispherical end whose lowest point (the tip) is at
// height zt, every point within rp of the axis above zt + rp.  Its surface
// point nearest to the sphere's centre lies on the line from the centre to
// the nearest axis point, (0, 0, max(z, zt + rp)), at distance d - rp.
// Returns the overlap R - (d - rp) and the unit vector n from the centre
// towards the axis point (no contact when the centre lies on the axis).
__device__ __forceinline__ double tool_overlap(double x, double y, double z, double R, double rp, double zt,
                                               double n[3]) {
  const double zc = __dadd_rn(zt, rp);
  const double az = z > zc ? z : zc;
  const double dz = __dsub_rn(az, z);
  const double d = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(dz, dz)));
  n[0] = n[1] = n[2] = 0.0;
  if (!(d > 0.0)) return -1.0;
  n[0] = __ddiv_rn(-x, d);
  n[1] = __ddiv_rn(-y, d);
  n[2] = __ddiv_rn(dz, d);
  return __dsub_rn(R, __dsub_rn(d, rp));
}

// One Hertz contact of a sphere with a flat or curved wall moving at vw
// along z: overlap delta, unit normal n from the centre towards the wall,
// spring history h (cleared when the contact has ended).  Returns the force
// on the sphere along z (0 without contact) and adds force and torque.
template <typename T, typename H>
__device__ __forceinline__ T wall_hertz(double delta, V3<T> n, double vw, const SampleDev& s, V3<T> v,
                                        V3<T> w, T R, T m, T Es, T Gs, T beta, T mu, T dt, H* h,
                                        V3<T>& F, V3<T>& Tq) {
  const H h0 = *h;
  V3<T> hist = v3<T>(h0.x, h0.y, h0.z);
  if (!(delta > 0.0)) {
    if (hist.x != T(0) || hist.y != T(0) || hist.z != T(0)) {
      H z;
      z.x = 0; z.y = 0; z.z = 0; z.w = 0;
      *h = z;
    }
    return T(0);
  }
  V3<T> vrel = v3<T>(-v.x, -v.y, T(vw) - v.z);
  V3<T> rw = v3<T>(R * w.x, R * w.y, R * w.z);
  V3<T> rwn = cross3(rw, n);
  V3<T> vc = v3<T>(vrel.x - rwn.x, vrel.y - rwn.y, vrel.z - rwn.z);
  V3<T> Fi, Ft;
  contact_law<T>(T(delta), n, vrel, vc, R, m, T(0), false, Es, Gs, beta, mu, dt, s.coulomb_mode,
                 hist, Fi, Ft);
  H hn;
  hn.x = hist.x; hn.y = hist.y; hn.z = hist.z; hn.w = 0;
  *h = hn;
  V3<T> nFt = cross3(n, Ft);
  F.x += Fi.x;
  F.y += Fi.y;
  F.z += Fi.z;
  Tq.x += R * nFt.x;
  Tq.y += R * nFt.y;
  Tq.z += R * nFt.z;
  return Fi.z;
}

// The penetrometer's contact, out of line: only the few spheres near an
// active tool take it, and inline it would cost every sphere registers.
template <typename T, typename H>
__device__ __noinline__ void tool_contact(const SampleDev& s, StageDev* W, double4 P, double r, V3<T> v,
                                          V3<T> w, T R, T m, T Es, T Gs, T beta, T mu, T dt, H* h,
                                          V3<T>* F, V3<T>* Tq) {
  double nd[3];
  (void)r;
  const double delta = tool_overlap(P.x, P.y, P.z, fabs(P.w), W->pen_radius, W->pen_z, nd);
  V3<T> Fl = *F, Tl = *Tq;
  const T fz = wall_hertz<T, H>(delta, v3<T>(T(nd[0]), T(nd[1]), T(nd[2])),
                                W->v_pen, s, v, w, R, m, Es, Gs, beta, mu, dt,
                                h, Fl, Tl);
  *F = Fl;
  *Tq = Tl;
  if (delta > 0.0)  // the sphere pushes the tool with -F
    atomicAdd(&W->pen_q, (unsigned long long)__double2ll_rn(-(double)fz * 1099511627776.0));
}

// Wall contacts of the cylinder (Sec. 3.1: Hertz particle-wall law): the
// side, the bottom (open over the outlet), the top plate and the
// penetrometer of a preparation stage, the last two moving along z (their
// velocity enters the contact's relative velocity).  A float pre-check
// selects the walls within 5 % of the radius; only those load their spring
// history and compute the overlap in FP64.  A sphere cannot move 5 % of its
// radius relative to a wall in one step (the boundaries move by v dt), so
// every wall with a non-zero history is among them (and gets its history
// cleared when the contact ends).  The forces the sphere exerts on the plate
// and the penetrometer along z are summed in integer quanta of 2^-40 N.
template <typename T, typename H, bool PREP>
__device__ __forceinline__ void wall_contacts(const SampleDev& s, StageDev& W, double4 P, float xf,
                                              float yf, float zf, V3<T> v, V3<T> w, T R, T m, T Es, T Gs,
                                              T beta, T mu, T dt, H* hist_base, size_t stride,
                                              V3<T>& F, V3<T>& Tq) {
  const float Rf = (float)R;
  const float rf = sqrtf(xf * xf + yf * yf);
  const float near = -0.05f * Rf;
  const double Hw = PREP ? W.H : s.H;
  const bool closed = PREP && W.outlet_closed;
  float dw[3] = {rf + Rf - s.Rc_f, (closed || rf >= s.r_out_f * 0.999f) ? Rf - zf : -1e30f,
                 zf + Rf - (PREP ? (float)Hw : s.H_f)};
  bool tool = false;
  if (PREP && W.pen_dir != 0) {
    const float rp = (float)W.pen_radius, zc = (float)W.pen_z + rp;
    const float dz = zf > zc ? 0.f : zc - zf;
    tool = Rf + rp - sqrtf(rf * rf + dz * dz) > near;
  }
  // most spheres are far from every wall: leave before any FP64 work (the
  // compiler would otherwise hoist the loop-invariant radius and its square
  // root out of the wall loop and run them for every sphere)
  if (!(dw[0] > near) && !(dw[1] > near) && !(dw[2] > near) && !tool) return;
  const double r2 = __dadd_rn(__dmul_rn(P.x, P.x), __dmul_rn(P.y, P.y));
  for (int wall = 0; wall < 3; ++wall) {
    if (!(dw[wall] > near)) continue;
    double delta = -1.0;
    double vw = 0.0;  // the wall's velocity along z
    V3<T> n = v3<T>(0, 0, 0);
    if (wall == 0) {
      if (r2 > 0.0) {
        const double r = sqrt(r2);
        delta = (r + fabs(P.w)) - s.Rc;
        n = v3<T>(T(P.x / r), T(P.y / r), T(0));
      }
    } else if (wall == 1) {
      if (P.z < fabs(P.w) && (closed || sqrt(r2) >= s.r_out)) {
        delta = fabs(P.w) - P.z;
        n = v3<T>(0, 0, -1);
      }
    } else {
      delta = (P.z + fabs(P.w)) - Hw;
      n = v3<T>(0, 0, 1);
      if (PREP) vw = W.v_plate;
    }
    const T fz = wall_hertz<T, H>(delta, n, vw, s, v, w, R, m, Es, Gs, beta, mu, dt,
                                  hist_base + (size_t)wall * stride, F, Tq);
    if (PREP && wall == 2 && delta > 0.0)  // the sphere pushes the plate with -F
      atomicAdd(&W.plate_q, (unsigned long long)__double2ll_rn(-(double)fz * 1099511627776.0));
  }
  if (PREP && tool)
    tool_contact<T, H>(s, &W, P, sqrt(r2), v, w, R, m, Es, Gs, beta, mu, dt, hist_base + 3 * stride, &F, &Tq);
}

// Fluid cell of a position with a float pre-check: the FP64 evaluation of
// floor((x - lo) * inv_h) is needed only within 1e-4 cell of a cell face.
__device__ __forceinline__ int fluid_cell_fast(const SampleDev& S, double x, double y, double z,
                                               float xf, float yf, float zf) {
  const float pf[3] = {xf, yf, zf};
  int c[3];
  bool exact = false;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float t = (pf[k] - S.f_lo_f[k]) * S.inv_hf_f[k];
    const float fl = floorf(t);
    const float fr = t - fl;
    if (!(fr >= 1e-4f && fr <= 1.f - 1e-4f)) exact = true;  // near a face, or not finite
    int ck = (int)fl;
    if (ck < 0) ck = 0;
    if (ck > S.nf[k] - 1) ck = S.nf[k] - 1;
    c[k] = ck;
  }
  if (exact) return fluid_cell_of(S, x, y, z);
  return S.fcell_off + (c[2] * S.nf[1] + c[1]) * S.nf[0] + c[0];
}

// ---- learned closure: the network's forward pass on the tensor cores ----

// all threads wait for the MMA group committed on bar; false on timeout
__device__ __forceinline__ bool cl_wait(uint64_t* bar, uint32_t& phase) {
  const bool ok = tc05::mbar_wait(bar, phase);
  phase ^= 1u;
  const int bad = __syncthreads_or(!ok);
  tc05::fence_after_sync();
  return bad == 0;
}
__device__ __forceinline__ void cl_publish() {
  tc05::fence_smem_to_async();
  tc05::fence_before_sync();
  __syncthreads();
  tc05::fence_after_sync();
}

// One forward pass over the block's 128 rows (thread t = row t, M = 128):
// x_hat = (f - mu) inv_sigma, three SiLU layers of 64 and the 2 outputs,
// BF16 operands from shared memory, FP32 accumulators in 64 TMEM columns.
// sm holds the network blob (bulk copy completing on bar[0]); bar[1] tracks
// the MMAs.  False (in every thread) if a bounded wait expired.
__device__ bool closure_infer(const float (&f)[5], uint8_t* sm, uint64_t* bar, uint32_t tb, float& o0,
                              float& o1) {
  using namespace tc05;
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t s0 = smem_u32(sm);
  const bool got = mbar_wait(&bar[0], 0);
  if (__syncthreads_or(!got)) return false;
  const float* P = reinterpret_cast<const float*>(sm + CL_TILES);
  float xh[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) xh[k] = (f[k] - P[CL_P_MU + k]) * P[CL_P_ISG + k];
  *reinterpret_cast<uint4*>(sm + CL_SM_A0 + tile_off(tid, 0, 16)) =
      make_uint4(pack_bf16x2(xh[0], xh[1]), pack_bf16x2(xh[2], xh[3]), pack_bf16x2(xh[4], 0.0f), 0u);
  *reinterpret_cast<uint4*>(sm + CL_SM_A0 + tile_off(tid, 8, 16)) = make_uint4(0u, 0u, 0u, 0u);
  cl_publish();
  uint32_t ph = 0;
  const uint32_t ID64 = idesc_bf16(128, 64), ID16 = idesc_bf16(128, 16);
  if (tid == 0) {
    mma_bf16(tb, kdesc(s0 + CL_SM_A0, 16, 0), kdesc(s0, 16, 0), ID64, 0u);
    mma_commit(&bar[1]);
  }
#pragma unroll 1
  for (int l = 0; l < 3; ++l) {
    if (!cl_wait(&bar[1], ph)) return false;
    const float* bias = P + CL_P_B1 + 64 * l;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float z[16];
      tmem_ld16(taddr(tb, 32u * warp, 16u * c), z);
      float h[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float zz = z[j] + bias[16 * c + j];
        h[j] = __fdividef(zz, 1.0f + __expf(-zz));  // SiLU; 0 where the exponential overflows
      }
#pragma unroll
      for (int hf = 0; hf < 2; ++hf)
        *reinterpret_cast<uint4*>(sm + CL_SM_AH + tile_off(tid, 16 * c + 8 * hf, 64)) =
            make_uint4(pack_bf16x2(h[8 * hf + 0], h[8 * hf + 1]), pack_bf16x2(h[8 * hf + 2], h[8 * hf + 3]),
                       pack_bf16x2(h[8 * hf + 4], h[8 * hf + 5]), pack_bf16x2(h[8 * hf + 6], h[8 * hf + 7]));
    }
    cl_publish();
    if (tid == 0) {
      const uint32_t w = l == 0 ? 2048u : (l == 1 ? 10240u : 18432u);
      for (uint32_t s = 0; s < 4; ++s)
        mma_bf16(tb, kdesc(s0 + CL_SM_AH, 64, s), kdesc(s0 + w, 64, s), l < 2 ? ID64 : ID16, s > 0);
      mma_commit(&bar[1]);
    }
  }
  if (!cl_wait(&bar[1], ph)) return false;
  float v[16];
  tmem_ld16(taddr(tb, 32u * warp, 0u), v);
  o0 = v[0] + P[CL_P_B4];
  o1 = v[1] + P[CL_P_B4 + 1];
  return true;
}

// Data of the particle that owns a record, broadcast to the lane evaluating it.
template <bool MIXED>
struct Owner;
template <>
struct Owner<true> {
  int4 pq;    // fixed-point position, fixed-point radius
  float4 va;  // v, R
  float4 wa;  // w, m
};
template <>
struct Owner<false> {
  double4 P, V, W;  // x,R | v,1/m | w,1/I
};

// The per-sphere end of a step, shared by both force kernels: walls,
// gravity, buoyancy, drag, velocity Verlet, fixed-point shadows, porosity
// scatter, closure network, and the step's bookkeeping (displacement since
// the rebuild, porosity rotation, step counter, next rebuild condition).
// valid: this thread owns sphere p (of sample si) and ends its step; F, Tq
// and the closure sums hold its contact forces.
template <bool MIXED, int MODE, bool CL, bool PREP>
__device__ __forceinline__ void finish_step(
    const Dev& d, Ctl* ctl, int cur, int nxt, int pc, int vfc, long long m_step, bool couple_next,
    uint32_t epoch, int lane, bool valid, int p, int si, const Owner<MIXED>& me,
    V3<typename std::conditional<MIXED, float, double>::type> F,
    V3<typename std::conditional<MIXED, float, double>::type> Tq,
    typename std::conditional<MIXED, float, double>::type Zacc,
    typename std::conditional<MIXED, float, double>::type Dacc,
    typename std::conditional<MIXED, float, double>::type Cacc, float2 my_c, bool use_c, bool feat,
    bool rec, bool net, uint8_t* cl_sm, uint64_t* cl_bar, uint32_t cl_tmem, unsigned* bk_n, int* bk_s,
    float* bk_m, unsigned* bk_c, cudaGraphConditionalHandle h_next,
    cudaGraphConditionalHandle h_fluid) {
  using T = typename std::conditional<MIXED, float, double>::type;
  // ---- per-particle epilogue: walls, body forces, drag, integration ----
  float my_disp2 = -1.f;
  bool coupled = false;
  float ft[5] = {0.f, 0.f, 0.f, 0.f, 0.f};  // closure inputs of this particle
  bool net_row = false;
  if (rec && valid) {  // inactive particles record zeros
    float4* r4 = reinterpret_cast<float4*>(d.clrec + (size_t)p * CL_COLS);
    r4[0] = make_float4(0.f, 0.f, 0.f, 0.f);
    r4[1] = make_float4(0.f, 0.f, 0.f, 0.f);
    r4[2] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (valid) {
    const SampleDev& S = d.sp[si];
    double4 P;
    if constexpr (MIXED) P = d.pos[cur][p];
    else P = me.P;
    const int fc0 = d.fcell[pc][p];
    if (S.use_drag) {
      prefetch_l1(&d.vf[vfc][fc0]);
      prefetch_l1(MIXED ? (const void*)&d.Usf[fc0] : (const void*)&d.Us[fc0]);
    }
    const bool active = P.w > 0.0;
    if (!active) {
      if (MODE != MODE_FORCES) {
        d.pos[nxt][p] = P;
        d.vel[nxt][p] = d.vel[cur][p];
        d.omg[nxt][p] = d.omg[cur][p];
        d.posq[nxt][p] = d.posq[cur][p];
        d.velf[nxt][p] = d.velf[cur][p];
        d.omgf[nxt][p] = d.omgf[cur][p];
      }
      if (MODE != MODE_MID) {
        d.F[p] = make_double4(0, 0, 0, 0);
        d.T[p] = make_double4(0, 0, 0, 0);
      }
    } else {
      double4 Vd, Wd;
      T Ri, mi;
      V3<T> vi, wi;
      if constexpr (MIXED) {
        Vd = d.vel[cur][p];
        Wd = d.omg[cur][p];
        vi = v3<T>(me.va.x, me.va.y, me.va.z);
        wi = v3<T>(me.wa.x, me.wa.y, me.wa.z);
        Ri = me.va.w;
        mi = me.wa.w;
      } else {
        Vd = me.V;
        Wd = me.W;
        vi = v3<T>(Vd.x, Vd.y, Vd.z);
        wi = v3<T>(Wd.x, Wd.y, Wd.z);
        Ri = P.w;
        mi = 1.0 / Vd.w;
      }
      const float xf = __double2float_rn(P.x), yf = __double2float_rn(P.y), zf = __double2float_rn(P.z);
      T Es, Gs, beta, mu, dt;
      if constexpr (MIXED) {
        Es = S.Es_f; Gs = S.Gs_f; beta = S.beta_f; mu = S.mu_f32; dt = S.dt_f;
      } else {
        Es = S.Es; Gs = S.Gs; beta = S.beta; mu = S.mu; dt = S.dt;
      }
      if (S.kind == CGDEM_CYLINDER) {
        if constexpr (MIXED)
          wall_contacts<T, float4, PREP>(S, d.stage[si], P, xf, yf, zf, vi, wi, Ri, mi, Es, Gs, beta, mu, dt,
                                   d.wallhf[pc] + p, (size_t)d.Npad, F, Tq);
        else
          wall_contacts<T, double4, PREP>(S, d.stage[si], P, xf, yf, zf, vi, wi, Ri, mi, Es, Gs, beta, mu, dt,
                                    d.wallh[pc] + p, (size_t)d.Npad, F, Tq);
      }
      // gravity, buoyancy (Eq. 1) and drag (Eq. 8-11)
      {
        T rho_s, rf, g0, g1, g2, nmin, muf;
        if constexpr (MIXED) {
          rho_s = S.rho_s_f; rf = S.rho_f32; g0 = S.g_f[0]; g1 = S.g_f[1]; g2 = S.g_f[2];
          nmin = S.n_min_f; muf = S.muf_f32;
        } else {
          rho_s = S.rho; rf = S.rho_f; g0 = S.g[0]; g1 = S.g[1]; g2 = S.g[2];
          nmin = S.n_min; muf = S.mu_f;
        }
        const T Vp = mi / rho_s;
        F.x += mi * g0;
        F.y += mi * g1;
        F.z += mi * g2;
        if (S.use_buoyancy) {
          F.x -= rf * Vp * g0;
          F.y -= rf * Vp * g1;
          F.z -= rf * Vp * g2;
        }
        if (S.use_drag || feat) {
          const int fc = fc0;
          const unsigned long long Sc = d.vf[vfc][fc];
          T scount;
          if constexpr (MIXED) scount = u64_to_f(Sc);
          else scount = (double)Sc;
          T nc = T(1) - scount * T(9.094947017729282379150390625e-13);  // 2^-40
          if (nc < nmin) nc = nmin;
          if (nc > T(1)) nc = T(1);
          V3<T> U;
          if constexpr (MIXED) {
            const float4 u = d.Usf[fc];
            U = v3<T>(u.x, u.y, u.z);
          } else {
            const double4 u = d.Us[fc];
            U = v3<T>(u.x, u.y, u.z);
          }
          const V3<T> w = v3<T>(U.x / nc - vi.x, U.y / nc - vi.y, U.z / nc - vi.z);
          V3<T> fd = v3<T>(0, 0, 0);
          if (S.use_drag) {
            fd = drag_force<T>(rf, muf, T(2) * Ri, w, nc);
            if (use_c) {  // drag correction of the closure
              fd.x *= (T)my_c.x;
              fd.y *= (T)my_c.x;
              fd.z *= (T)my_c.x;
            }
            F.x += fd.x;
            F.y += fd.y;
            F.z += fd.z;
          }
          if (S.fluid_mode == 1 && d.any_fluid) {
            // Darcy flow: the dynamic pressure gradient on the grain's volume,
            // and the drag's reaction on the fluid (Eq. 7) summed per cell in
            // integer quanta of 2^-60 N, into the buffer of this evaluation
            V3<T> G;
            if constexpr (MIXED) {
              const float4 g = d.gradpf[fc];
              G = v3<T>(g.x, g.y, g.z);
            } else {
              const double4 g = d.gradp[fc];
              G = v3<T>(g.x, g.y, g.z);
            }
            F.x -= Vp * G.x;
            F.y -= Vp * G.y;
            F.z -= Vp * G.z;
            if (MODE != MODE_MID) {
              // only an evaluation that ends a call can be read back
              // (cgdem_get_fluid): a step inside a call sums no reaction
              const long long e = MODE == MODE_FORCES ? m_step - 1 : m_step;
              unsigned long long* rx = d.react[e & 1] + 3 * (size_t)fc;
              atomicAdd(rx, (unsigned long long)__double2ll_rn((double)fd.x * 1152921504606846976.0));
              atomicAdd(rx + 1, (unsigned long long)__double2ll_rn((double)fd.y * 1152921504606846976.0));
              atomicAdd(rx + 2, (unsigned long long)__double2ll_rn((double)fd.z * 1152921504606846976.0));
            }
          }
          if (feat) {
            net_row = true;
            ft[0] = (float)(T(1) - nc);
            ft[1] = (float)m_sqrt(dot3(w, w));
            ft[2] = S.k_feat_f;
            ft[3] = (float)Zacc;
            ft[4] = Zacc > T(0) ? (float)(Dacc / (Zacc * T(2) * Ri)) : 0.f;
            if (rec) {
              float4* r4 = reinterpret_cast<float4*>(d.clrec + (size_t)p * CL_COLS);
              r4[0] = make_float4(ft[0], ft[1], ft[2], ft[3]);
              r4[1] = make_float4(ft[4], (float)fd.x, (float)fd.y, (float)fd.z);
              r4[2] = make_float4((float)Cacc, (float)(fc - S.fcell_off), my_c.x, my_c.y);
            }
          }
        }
      }
      if (!isfinite(F.x + F.y + F.z + Tq.x + Tq.y + Tq.z)) latch(ctl, ST_NONFINITE);

      if (MODE == MODE_FORCES) {
        d.F[p] = make_double4((double)F.x, (double)F.y, (double)F.z, 0.0);
        d.T[p] = make_double4((double)Tq.x, (double)Tq.y, (double)Tq.z, 0.0);
      } else {
        // outlet (produced sand, Eq. 40): float filter, FP64 decision
        const bool removed = S.kind == CGDEM_CYLINDER && zf < -1.999f * __double2float_rn(P.w) &&
                             P.z < -2.0 * P.w;
        if (removed) {
          d.removed_step[d.id[pc][p]] = (int)m_step;
          record_produced(d, S, si, P.w);
        }
        double vx, vy, vz, wx, wy, wz;
        if constexpr (MIXED) {
          // FP32 force increments added to the FP64 state
          const float im = 1.0f / me.wa.w;
          const float iI = __double2float_rn(Wd.w);
          const float c = (MODE == MODE_MID ? S.dt_f : 0.5f * S.dt_f);
          vx = Vd.x + (double)(c * im * (float)F.x);
          vy = Vd.y + (double)(c * im * (float)F.y);
          vz = Vd.z + (double)(c * im * (float)F.z);
          wx = Wd.x + (double)(c * iI * (float)Tq.x);
          wy = Wd.y + (double)(c * iI * (float)Tq.y);
          wz = Wd.z + (double)(c * iI * (float)Tq.z);
        } else {
          const double h = S.half_dt, im = Vd.w, iI = Wd.w;
          vx = Vd.x + h * (F.x * im);
          vy = Vd.y + h * (F.y * im);
          vz = Vd.z + h * (F.z * im);
          wx = Wd.x + h * (Tq.x * iI);
          wy = Wd.y + h * (Tq.y * iI);
          wz = Wd.z + h * (Tq.z * iI);
          if (MODE == MODE_MID) {
            vx += h * (F.x * im);
            vy += h * (F.y * im);
            vz += h * (F.z * im);
            wx += h * (Tq.x * iI);
            wy += h * (Tq.y * iI);
            wz += h * (Tq.z * iI);
          }
        }
        if (MODE == MODE_CANON) {
          d.F[p] = make_double4((double)F.x, (double)F.y, (double)F.z, 0.0);
          d.T[p] = make_double4((double)Tq.x, (double)Tq.y, (double)Tq.z, 0.0);
          double4 Pn = P;
          int4 pqn = d.posq[cur][p];
          if (removed) {
            Pn.w = -P.w;
            pqn.w = 0;
          }
          d.pos[nxt][p] = Pn;
          d.vel[nxt][p] = make_double4(vx, vy, vz, Vd.w);
          d.omg[nxt][p] = make_double4(wx, wy, wz, Wd.w);
          d.posq[nxt][p] = pqn;
          const float4 va = d.velf[cur][p], wa = d.omgf[cur][p];
          d.velf[nxt][p] = make_float4(__double2float_rn(vx), __double2float_rn(vy), __double2float_rn(vz), va.w);
          d.omgf[nxt][p] = make_float4(__double2float_rn(wx), __double2float_rn(wy), __double2float_rn(wz), wa.w);
        } else if (removed) {
          double4 Pn = P;
          Pn.w = -P.w;
          d.pos[nxt][p] = Pn;
          d.vel[nxt][p] = Vd;
          d.omg[nxt][p] = Wd;
          int4 pqn = d.posq[cur][p];
          pqn.w = 0;
          d.posq[nxt][p] = pqn;
          d.velf[nxt][p] = d.velf[cur][p];
          d.omgf[nxt][p] = d.omgf[cur][p];
        } else {
          double x = P.x + S.dt * vx, y = P.y + S.dt * vy, z = P.z + S.dt * vz;
          float nxf = __double2float_rn(x), nyf = __double2float_rn(y), nzf = __double2float_rn(z);
          if (S.kind == CGDEM_PERIODIC_BOX) {
            const float Lf = S.L_f[0], eps = 1e-4f * Lf;
            if (nxf < eps || nxf > Lf - eps) {
              if (x >= S.L[0]) x -= S.L[0]; else if (x < 0.0) x += S.L[0];
              nxf = __double2float_rn(x);
            }
            if (nyf < eps || nyf > Lf - eps) {
              if (y >= S.L[1]) y -= S.L[1]; else if (y < 0.0) y += S.L[1];
              nyf = __double2float_rn(y);
            }
            if (nzf < eps || nzf > Lf - eps) {
              if (z >= S.L[2]) z -= S.L[2]; else if (z < 0.0) z += S.L[2];
              nzf = __double2float_rn(z);
            }
          }
          d.pos[nxt][p] = make_double4(x, y, z, P.w);
          d.vel[nxt][p] = make_double4(vx, vy, vz, Vd.w);
          d.omg[nxt][p] = make_double4(wx, wy, wz, Wd.w);
          int4 pqn;
          if (S.q_exp != 0x7fffffff) {
            pqn.x = to_q_pow2(x, S.q_exp);
            pqn.y = to_q_pow2(y, S.q_exp);
            pqn.z = to_q_pow2(z, S.q_exp);
          } else {
            pqn.x = to_q(x, S.inv_dq);
            pqn.y = to_q(y, S.inv_dq);
            pqn.z = to_q(z, S.inv_dq);
          }
          float Rf, mf;
          if constexpr (MIXED) {
            pqn.w = me.pq.w;
            Rf = me.va.w;
            mf = me.wa.w;
          } else {
            pqn.w = d.posq[cur][p].w;
            Rf = d.velf[cur][p].w;
            mf = d.omgf[cur][p].w;
          }
          d.posq[nxt][p] = pqn;
          d.velf[nxt][p] = make_float4(__double2float_rn(vx), __double2float_rn(vy), __double2float_rn(vz), Rf);
          d.omgf[nxt][p] = make_float4(__double2float_rn(wx), __double2float_rn(wy), __double2float_rn(wz), mf);
          const int4 ref = d.posq_ref[p];
          const float ex = (float)(int)((uint32_t)pqn.x - (uint32_t)ref.x);
          const float ey = (float)(int)((uint32_t)pqn.y - (uint32_t)ref.y);
          const float ez = (float)(int)((uint32_t)pqn.z - (uint32_t)ref.z);
          my_disp2 = ex * ex + ey * ey + ez * ez;
          const int fc = fluid_cell_fast(S, x, y, z, nxf, nyf, nzf);
          d.fcell[pc][p] = fc;
          if (couple_next) {
            coupled = true;
            if (S.vf_mode == 0) atomicAdd(&d.vf[(vfc + 1) % 3][fc], d.vq[pc][p]);
          }
        }
      }
    }
  }

  // ---- learned closure: corrections for the next evaluation ----
  if (net) {
    float o0 = 0.f, o1 = 0.f;
    const bool ok = closure_infer(ft, cl_sm, cl_bar, cl_tmem, o0, o1);
    if (valid) {
      float2 c = make_float2(1.0f, 1.0f);  // plain coarse-graining outside the training range
      if (ok && net_row) {
        const float* P = reinterpret_cast<const float*>(cl_sm + CL_TILES);
        bool inside = true;
#pragma unroll
        for (int k = 0; k < 5; ++k) inside = inside && ft[k] >= P[CL_P_LO + k] && ft[k] <= P[CL_P_HI + k];
        if (inside) {
          const float cdm = P[CL_P_CMAX], cgm = P[CL_P_CMAX + 1];
          c.x = expf(fminf(fmaxf(o0, -cdm), cdm));
          c.y = expf(fminf(fmaxf(o1, -cgm), cgm));
        }
      }
      d.clc[nxt][p] = c;
    }
    if (!ok && threadIdx.x == 0) latch(ctl, ST_TIMEOUT);
    tc05::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tc05::tmem_dealloc(cl_tmem, 64);
  }

  // ---- bookkeeping: displacement since rebuild, porosity rotation, step ----
  const int wib = threadIdx.x >> 5;
  if (d.any_fluid) {  // the next evaluation's reaction buffer starts at zero
    const long long e = MODE == MODE_FORCES ? m_step - 1 : m_step;
    unsigned long long* z = d.react[(e + 1) & 1];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < 3 * d.Cf_total; c += gridDim.x * blockDim.x)
      z[c] = 0ull;
  }
  if (MODE == MODE_MID) {
    unsigned long long* z = d.vf[(vfc + 2) % 3];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < d.Cf_total; c += gridDim.x * blockDim.x)
      z[c] = 0ull;
    const int s0 = __shfl_sync(FULL, si, 0);
    const bool uniform = __all_sync(FULL, !valid || si == s0);
    float md = my_disp2;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) md = fmaxf(md, __shfl_xor_sync(FULL, md, o));
    // one fence and one arrival per block, without a block barrier: each
    // warp leaves its maximum in shared memory, and the block's last warp
    // publishes them (a warp that straddles samples publishes per lane and
    // fences)
    const unsigned wcoupled = __any_sync(FULL, coupled) ? 1u : 0u;
    if (!uniform) {
      if (my_disp2 >= 0.f) atomicMax(&d.dmax2[si], __float_as_uint(my_disp2));
      __threadfence();
    }
    if (lane == 0) {
      bk_s[wib] = s0;
      bk_m[wib] = uniform ? md : -1.f;
      bk_c[wib] = wcoupled;
    }
  }
  if (lane != 0) return;
  __threadfence_block();
  const unsigned nw = blockDim.x >> 5;
  if (atomicAdd(bk_n, 1u) != nw - 1u) return;
  __threadfence_block();
  {
    if (MODE == MODE_MID) {
      unsigned any = 0u;
      for (unsigned w = 0; w < nw; ++w) {
        const float mw = *((volatile float*)&bk_m[w]);
        if (mw >= 0.f) atomicMax(&d.dmax2[*((volatile int*)&bk_s[w])], __float_as_uint(mw));
        any |= *((volatile unsigned*)&bk_c[w]);
      }
      if (any) atomicOr(&ctl->coupled, 1u);
    }
    __threadfence();
    const unsigned t = atomicAdd(&ctl->block_counter, 1u);
    if (t == gridDim.x - 1) {
      // every block has started and finished: the segment order and the
      // flags' epoch move on for the next launch
      __threadfence();
      if (MODE == MODE_MID) {
        for (int s = 0; s < d.n_samples; ++s) {
          const unsigned b = atomicAdd(&d.dmax2[s], 0u);
          if (__uint_as_float(b) > d.sp[s].rebuild_q2) ctl->rebuild = 1;
        }
        if (atomicExch(&ctl->coupled, 0u)) {
          ctl->vf_cur = (vfc + 1) % 3;
          ctl->fl_pending = 1;  // the Darcy flow follows the new porosity
        }
        ctl->cur = nxt;
        ctl->step = m_step;
      }
      // the moving boundaries: this evaluation's forces on them, the plate's
      // next velocity, and (a step that drifts the grains) their drift
      for (int s = 0; PREP && s < d.n_samples; ++s) {
        if (d.sp[s].kind != CGDEM_CYLINDER) continue;
        close_boundaries(d.stage[s], d.sp[s].Rc);
        if (MODE == MODE_MID) drift_boundaries(d.stage[s], d.sp[s].dt);
      }
      ctl->epoch = epoch;
      ctl->blk_next = 0;
      ctl->block_counter = 0u;
      __threadfence();
      if (MODE == MODE_MID && h_next) cudaGraphSetConditional(h_next, ctl->rebuild ? 1u : 0u);
      // the step's Darcy solve runs when this step updated the porosity
      if (MODE == MODE_MID && h_fluid) cudaGraphSetConditional(h_fluid, ctl->fl_pending ? 1u : 0u);
    }
  }
}

// FP64: each pair listed once, by its lower-index sphere.  Warps walk their
// record segment in rounds of 32 entries (every lane evaluates one pair per
// round whatever the list lengths are); each entry's owner is found by a
// search over the lanes and its data broadcast, and a round's contributions
// are summed per sphere by a segmented scan in list order.  The owner's warp
// passes the pair's result to the partner through the partner's inbox (see
// the file comment).  CL: the context carries the learned closure (blocks of
// 128 threads; more registers per thread for the closure data and the network
// epilogue).
// h_next: conditional handle of the next step's rebuild node when the launch
// sits in a CUDA graph (0 otherwise); h_fluid: that of the step's Darcy-solve
// node (0: none); the step's last warp sets both.
template <int MODE, bool CL, bool PREP>
__global__ void __launch_bounds__(CL ? 128 : FORCE_BLOCK_MAX, CL ? 5 : CGDEM_PAIRS_MINB)
    k_forces_pairs(Dev d, cudaGraphConditionalHandle h_next,
    cudaGraphConditionalHandle h_fluid) {
  using T = double;
  Ctl* ctl = d.ctl;
  const int cur = ctl->cur;
  const int nxt = cur ^ 1;
  const int pc = ctl->pcur;
  const int rc = ctl->rec_cur;
  const int vfc = ctl->vf_cur;
  const long long m_step = ctl->step + 1;  // step completed by this evaluation
  // porosity recomputed for the next positions (couple_every is equal in all samples)
  const int ce = d.sp[0].couple_every;
  const bool couple_next = ce == 1 || (unsigned)(m_step % ce) == 0u;
  const int lane = threadIdx.x & 31;
  // blocks take their segments in the order they start (a counter), so a
  // warp only ever waits for warps that are already running
  const uint32_t epoch = ctl->epoch + 1u;  // value of a segment flag once its pairs are done
  __shared__ int blk_s;
  __shared__ unsigned bk_n;
  if (threadIdx.x == 0) {
    blk_s = atomicAdd(&ctl->blk_next, 1);
    bk_n = 0u;
  }
  __syncthreads();
  // P spheres per warp (32; 16 for small samples, twice the warps to hide
  // latency); lanes >= P own no sphere but evaluate entries.  The grid
  // covers Npad / P warps exactly.
  const int P = d.ppw;
  const int sg = (blk_s * (int)blockDim.x + (int)threadIdx.x) >> 5;  // segment of this warp
  const int wbase = sg * P;
  const bool owner_lane = lane < P;
  const int p = owner_lane ? wbase + lane : wbase;
  const bool valid = owner_lane && p < d.N;

  // learned closure: corrections in use, network evaluated after the
  // forces (blocks of 128), per-particle data recorded
  const bool use_c = CL && ctl->closure != 0;
  const bool net = use_c && MODE != MODE_FORCES && d.cl_smem;
  const bool rec = CL && ctl->record != 0;
  const bool feat = net || rec;
  __shared__ __align__(8) uint64_t cl_bar[2];
  __shared__ uint32_t cl_tmem;
  extern __shared__ uint8_t cl_raw[];
  uint8_t* cl_sm = nullptr;
  if (net) {
    const uint32_t a = tc05::smem_u32(cl_raw);
    cl_sm = cl_raw + (((a + 1023u) & ~1023u) - a);
    if (threadIdx.x == 0) {
      tc05::mbar_init(&cl_bar[0], 1);
      tc05::mbar_init(&cl_bar[1], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // the weights arrive while the contacts are evaluated
      tc05::mbar_expect_tx(&cl_bar[0], CL_BLOB);
      tc05::bulk_g2s(cl_sm, d.clblob, CL_BLOB, &cl_bar[0]);
    }
    if (threadIdx.x < 32) {
      tc05::tmem_alloc(&cl_tmem, 64);
      tc05::tmem_relinquish();
    }
    tc05::fence_before_sync();
    __syncthreads();
    tc05::fence_after_sync();
  }
  float2 my_c = make_float2(1.0f, 1.0f);
  if (use_c && valid) my_c = d.clc[cur][p];
  // per-block bookkeeping of the fused step (see the end of the kernel)
  __shared__ int bk_s[FORCE_BLOCK_MAX / 32];
  __shared__ float bk_m[FORCE_BLOCK_MAX / 32];
  __shared__ unsigned bk_c[FORCE_BLOCK_MAX / 32];

  // ---- own particle, contact phase ----
  Owner<false> me;
  int si = 0;
  if (valid) si = d.sample[pc][p];
  if (valid) {
    me.P = d.pos[cur][p];
    me.V = d.vel[cur][p];
    me.W = d.omg[cur][p];
  } else {
    me.P = make_double4(0, 0, 0, 0);
    me.V = make_double4(0, 0, 0, 1);
    me.W = make_double4(0, 0, 0, 1);
  }

  const uint32_t ncnt = owner_lane ? d.cnt[rc][p] : 0u;
  const uint32_t seg = (uint32_t)wbase * (uint32_t)d.cap;
  const uint32_t lo0 = owner_lane ? d.roff[rc][p] - seg : 0u;
  const uint32_t total = __shfl_sync(FULL, lo0 + ncnt, P - 1);
  // a lane without a sphere starts its (empty) run at the end: never an owner
  const uint32_t lo = owner_lane ? lo0 : total;
  V3<T> F = v3<T>(0, 0, 0), Tq = v3<T>(0, 0, 0);
  T Zacc = 0, Dacc = 0, Cacc = 0;  // closure data: active contacts, summed overlap, bond capacity

  for (uint32_t base = 0; base < total; base += 32) {
    const uint32_t e = base + lane;
    const bool has = e < total;
    // owner lane: the last lane whose first entry is <= e
    int own = 0;
#pragma unroll
    for (int sft = 16; sft >= 1; sft >>= 1) {
      const int c = own + sft;
      const uint32_t loc = __shfl_sync(FULL, lo, c & 31);
      if (c < 32 && loc <= e) own = c;
    }
    const int os = __shfl_sync(FULL, si, own);
    const float o_cg = use_c ? __shfl_sync(FULL, my_c.y, own) : 1.0f;
    T e_z = 0, e_d = 0, e_c = 0;
    Owner<false> o;
    o.P.x = __shfl_sync(FULL, me.P.x, own);
    o.P.y = __shfl_sync(FULL, me.P.y, own);
    o.P.z = __shfl_sync(FULL, me.P.z, own);
    o.P.w = __shfl_sync(FULL, me.P.w, own);
    o.V.x = __shfl_sync(FULL, me.V.x, own);
    o.V.y = __shfl_sync(FULL, me.V.y, own);
    o.V.z = __shfl_sync(FULL, me.V.z, own);
    o.V.w = __shfl_sync(FULL, me.V.w, own);
    o.W.x = __shfl_sync(FULL, me.W.x, own);
    o.W.y = __shfl_sync(FULL, me.W.y, own);
    o.W.z = __shfl_sync(FULL, me.W.z, own);

    V3<T> Fc = v3<T>(0, 0, 0), Tc = v3<T>(0, 0, 0);
    if (has) {
      const SampleDev& S = d.sp[os];
      const size_t idx = (size_t)seg + e;
      const uint32_t slot = d.rslot[idx];  // the pair's slot in the partner's inbox
      const int owner_p = wbase + own;
      uint32_t pf;
      V3<T> xi;
      const RecD* rr = reinterpret_cast<const RecD*>(d.rec[rc]) + idx;
      const int4 h0 = *reinterpret_cast<const int4*>(rr);
      const double2 h1 = *(reinterpret_cast<const double2*>(rr) + 1);
      pf = (uint32_t)h0.x;
      xi = v3<T>(__hiloint2double(h0.w, h0.z), h1.x, h1.y);

      const int q = (int)(pf & REC_IDX);
      bool bonded = (pf & REC_BOND) != 0u;
      const bool had_state = (pf & (REC_BOND | REC_ACTIVE)) != 0u ||
                             ((dbits(xi.x) | dbits(xi.y) | dbits(xi.z)) & 0x7fffffffffffffffLL) != 0;
      bool act = false;
      const double4 Q = d.pos[cur][q];
      if (dbits(Q.w) > 0 && dbits(o.P.w) > 0) {
        double dx = __dsub_rn(Q.x, o.P.x), dy = __dsub_rn(Q.y, o.P.y), dz = __dsub_rn(Q.z, o.P.z);
        if (S.kind == CGDEM_PERIODIC_BOX) {
          dx = min_image(dx, S.L[0]);
          dy = min_image(dy, S.L[1]);
          dz = min_image(dz, S.L[2]);
        }
        const double d2 =
            __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        const double Sd = __dadd_rn(o.P.w, Q.w);
        const bool touching = dbits(d2) < dbits(__dmul_rn(Sd, Sd));  // both >= 0
        if (bonded || touching) {
          const double dist = sqrt(d2);
          const double Rs = __dmul_rn(o.P.w, Q.w) / __dadd_rn(o.P.w, Q.w);
          const double delta = __dsub_rn(Sd, dist);
          double gam_d = S.gamma;  // gamma sqrt(c_g,i c_g,j) under the closure
          const bool orig_mode = PREP && S.jkr_mode == 1;
          if (use_c && (bonded || orig_mode)) gam_d = S.gamma * sqrt((double)o_cg * (double)d.clc[cur][q].y);
          const bool orig = orig_mode && gam_d > 0.0;
          if (bonded) {  // modified JKR: break at C for good; original JKR: separation at S
            if (orig ? contact_separates_exact(delta, Rs, S.Es, gam_d) : bond_breaks_exact(delta, Rs, S.Es, gam_d))
              bonded = false;
          } else if (orig && touching) {
            bonded = true;  // original JKR: the contact forms at A
          }
          act = bonded || touching;
          if (act && dbits(dist) > 0) {
            const double4 QV = d.vel[cur][q];
            const double4 QW = d.omg[cur][q];
            const double Ri = o.P.w, Rj = Q.w;
            const double idist = nr_rcp(dist);  // one reciprocal instead of three divisions
            const V3<double> n = v3<double>(dx * idist, dy * idist, dz * idist);
            // m* = m_i m_j / (m_i + m_j) = 1 / (1/m_i + 1/m_j), from the stored 1/m
            const double ms = nr_rcp(o.V.w + QV.w);
            const V3<double> vrel = v3<double>(QV.x - o.V.x, QV.y - o.V.y, QV.z - o.V.z);
            const V3<double> rw = v3<double>(Ri * o.W.x + Rj * QW.x, Ri * o.W.y + Rj * QW.y,
                                             Ri * o.W.z + Rj * QW.z);
            const V3<double> rwn = cross3(rw, n);
            const V3<double> vc = v3<double>(vrel.x - rwn.x, vrel.y - rwn.y, vrel.z - rwn.z);
            V3<double> Fi, Ft;
            V3<double> xid = v3<double>((double)xi.x, (double)xi.y, (double)xi.z);
            if (orig)  // the original JKR's branch down to S (preparation stages)
              contact_law<double>(delta, n, vrel, vc, Rs, ms, gam_d, bonded, S.Es, S.Gs, S.beta,
                                  S.mu, S.dt, S.coulomb_mode, xid, Fi, Ft, orig);
            else
              contact_law_fp64(delta, n, vrel, vc, Rs, ms, gam_d, bonded, S, xid, Fi, Ft);
            xi = v3<T>(xid.x, xid.y, xid.z);
            const V3<double> nFt = cross3(n, Ft);
            Fc = v3<T>(Fi.x, Fi.y, Fi.z);
            Tc = v3<T>(nFt.x, nFt.y, nFt.z);
            if (feat) {
              e_z = 1;
              e_d = delta;
              e_c = bonded ? 0.5 * 3.0 * PI_D * gam_d * Rs : 0.0;
            }
          } else if (act) {
            act = false;  // coincident centres: no normal defined
          }
        }
      }

      // write the record back when its state changed
      if (act) {
        const uint32_t npf = (uint32_t)q | REC_ACTIVE | (bonded ? REC_BOND : 0u);
        RecD* rr = reinterpret_cast<RecD*>(d.rec[rc]) + idx;
        const double xx = (double)xi.x;
        *reinterpret_cast<int4*>(rr) = make_int4((int)npf, 0, __double2loint(xx), __double2hiint(xx));
        *(reinterpret_cast<double2*>(rr) + 1) = make_double2((double)xi.y, (double)xi.z);

      } else if (had_state) {
        RecD* rr = reinterpret_cast<RecD*>(d.rec[rc]) + idx;
        *reinterpret_cast<int4*>(rr) = make_int4(q, 0, 0, 0);
        *(reinterpret_cast<double2*>(rr) + 1) = make_double2(0.0, 0.0);

      }
      // FP64: the pair's result for the partner (zeros when inactive), into
      // its slot of the partner's inbox: the force on the owner and n x F_t
      // (the torque on either sphere divided by its radius)
      {
        if (slot < (uint32_t)d.cap) {
          const size_t ib = (size_t)slot * d.Npad + q;
          double4* o4 = d.inbox + 2 * ib;
          o4[0] = make_double4(Fc.x, Fc.y, Fc.z, Tc.x);
          o4[1] = make_double4(Tc.y, Tc.z, 0.0, 0.0);
          if (feat) d.inbox_cl[ib] = make_float4((float)e_z, (float)e_d, (float)e_c, 0.f);
        }
      }
    }
    // contributions of this round to their owners: a segmented inclusive
    // scan over the lanes (entries of one owner are contiguous), then each
    // owner takes the value at the last lane of its run.  The tree order of
    // the sums is fixed by the list, so the result is deterministic.
    {
      const int key = has ? own : 32 + lane;
      T c0 = Fc.x, c1 = Fc.y, c2 = Fc.z, c3 = Tc.x, c4 = Tc.y, c5 = Tc.z;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int ku = __shfl_up_sync(FULL, key, off);
        const T u0 = __shfl_up_sync(FULL, c0, off);
        const T u1 = __shfl_up_sync(FULL, c1, off);
        const T u2 = __shfl_up_sync(FULL, c2, off);
        const T u3 = __shfl_up_sync(FULL, c3, off);
        const T u4 = __shfl_up_sync(FULL, c4, off);
        const T u5 = __shfl_up_sync(FULL, c5, off);
        if (lane >= off && ku == key) {
          c0 += u0;
          c1 += u1;
          c2 += u2;
          c3 += u3;
          c4 += u4;
          c5 += u5;
        }
      }
      const int a = (int)max(lo, base) - (int)base;
      const int b = (int)min(lo + ncnt, base + 32u) - (int)base;
      const int src = b > a ? b - 1 : 0;
      const T s0 = __shfl_sync(FULL, c0, src);
      const T s1 = __shfl_sync(FULL, c1, src);
      const T s2 = __shfl_sync(FULL, c2, src);
      const T s3 = __shfl_sync(FULL, c3, src);
      const T s4 = __shfl_sync(FULL, c4, src);
      const T s5 = __shfl_sync(FULL, c5, src);
      if (b > a) {
        F.x += s0;
        F.y += s1;
        F.z += s2;
        Tq.x += s3;
        Tq.y += s4;
        Tq.z += s5;
      }
      if (feat) {  // the closure data, same segments
        T c6 = e_z, c7 = e_d, c8 = e_c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const int ku = __shfl_up_sync(FULL, key, off);
          const T u6 = __shfl_up_sync(FULL, c6, off);
          const T u7 = __shfl_up_sync(FULL, c7, off);
          const T u8 = __shfl_up_sync(FULL, c8, off);
          if (lane >= off && ku == key) {
            c6 += u6;
            c7 += u7;
            c8 += u8;
          }
        }
        const T s6 = __shfl_sync(FULL, c6, src);
        const T s7 = __shfl_sync(FULL, c7, src);
        const T s8 = __shfl_sync(FULL, c8, src);
        if (b > a) {
          Zacc += s6;
          Dacc += s7;
          Cacc += s8;
        }
      }
    }
  }

  // ---- FP64: the pairs owned by lower-index partners ----
  // publish this segment, then wait for the segments owning the lowest
  // partners of its spheres (bounded: a wait that runs out reports a timeout)
  {
    __threadfence();
    __syncwarp();
    if (lane == 0) st_release_u32(&d.seg_flag[sg], epoch);
    const int w0 = (int)d.seg_wait[sg];
    bool ok = true;
    for (int t0 = w0; t0 < sg && ok; t0 += 32) {
      const int t = t0 + lane;
      for (int it = 0;; ++it) {
        const bool done = t >= sg || (int)(ld_acquire_u32(&d.seg_flag[t]) - epoch) >= 0;
        if (__all_sync(FULL, done)) break;
        if (it >= WAIT_LIMIT) {
          ok = false;
          break;
        }
        __nanosleep(64);
      }
    }
    if (!ok && lane == 0) latch(ctl, ST_TIMEOUT);
    __threadfence();
    if (valid) {
      // inbox in slot order: force on the owner negated, n x F_t as it is
      const uint32_t nin = d.inc_n[p];
#pragma unroll 4
      for (uint32_t k = 0; k < nin; ++k) {
        const double4* o4 = d.inbox + 2 * ((size_t)k * d.Npad + p);
        const double4 b0 = ldcg_d4(o4), b1 = ldcg_d4(o4 + 1);
        F.x -= b0.x;
        F.y -= b0.y;
        F.z -= b0.z;
        Tq.x += b0.w;
        Tq.y += b1.x;
        Tq.z += b1.y;
      }
      if (feat) {
        for (uint32_t k = 0; k < nin; ++k) {
          const float4 c = __ldcg(d.inbox_cl + (size_t)k * d.Npad + p);
          Zacc += c.x;
          Dacc += c.y;
          Cacc += c.z;
        }
      }
      // the torque arm R_i multiplies the summed n x F_t
      const T Ri = me.P.w;
      Tq = v3<T>(Ri * Tq.x, Ri * Tq.y, Ri * Tq.z);
    }
  }

  finish_step<false, MODE, CL, PREP>(d, ctl, cur, nxt, pc, vfc, m_step, couple_next, epoch, lane, valid, p, si, me,
                               F, Tq, Zacc, Dacc, Cacc, my_c, use_c, feat, rec, net, cl_sm, cl_bar, cl_tmem,
                               &bk_n, bk_s, bk_m, bk_c, h_next, h_fluid);
}


// Mixed precision: one lane per sphere (ppw = 32), or two lanes per sphere
// taking alternate entries of its list (ppw = 16, for samples too small to
// fill the GPU).  The rebuild orders the spheres of each tile of 1024
// consecutive spheres in cell order by candidate count and stores them in
// that order (the schedule order), so the spheres of a warp have lists of
// about the same length and are read and written in consecutive lines; a
// warp's records are stored entry-major (entry k of its lanes' spheres side
// by side), so every iteration of the loop below reads one contiguous line
// of records.  Each lane sums its own
// sphere's pairs in list order: no search for the owner of an entry, no
// broadcast of its data and no segmented scan, and the sums stay
// deterministic.
template <int MODE, bool CL, bool PREP>
__global__ void __launch_bounds__(CL ? 128 : FORCE_BLOCK_MAX, CL ? 5 : CGDEM_FORCE_MINB)
    k_forces_lanes(Dev d, cudaGraphConditionalHandle h_next,
    cudaGraphConditionalHandle h_fluid) {
  Ctl* ctl = d.ctl;
  const int cur = ctl->cur;
  const int nxt = cur ^ 1;
  const int pc = ctl->pcur;
  const int rc = ctl->rec_cur;
  const int vfc = ctl->vf_cur;
  const long long m_step = ctl->step + 1;  // step completed by this evaluation
  const int ce = d.sp[0].couple_every;
  const bool couple_next = ce == 1 || (unsigned)(m_step % ce) == 0u;
  const int lane = threadIdx.x & 31;
  const uint32_t epoch = ctl->epoch + 1u;
  __shared__ unsigned bk_n;
  if (threadIdx.x == 0) bk_n = 0u;
  __syncthreads();
  const int P = d.ppw;                  // spheres per warp
  const int Lp = 32 / P;                // lanes per sphere (1 or 2)
  const int sub = lane & (P - 1);       // the warp's sphere this lane works on
  const int half = lane / P;            // which of its entries: half, half + Lp, ...
  const int gw = (blockIdx.x * (int)blockDim.x + (int)threadIdx.x) >> 5;
  const int slot = gw * P + sub;        // the grid covers Npad slots exactly
  const bool has = slot < d.N;
  const int p = has ? slot : 0;
  const bool valid = has && half == 0;  // the lane that ends the sphere's step

  // learned closure: corrections in use, network evaluated after the
  // forces (blocks of 128), per-particle data recorded
  const bool use_c = CL && ctl->closure != 0;
  const bool net = use_c && MODE != MODE_FORCES && d.cl_smem;
  const bool rec = CL && ctl->record != 0;
  const bool feat = net || rec;
  __shared__ __align__(8) uint64_t cl_bar[2];
  __shared__ uint32_t cl_tmem;
  extern __shared__ uint8_t cl_raw[];
  uint8_t* cl_sm = nullptr;
  if (net) {
    const uint32_t a = tc05::smem_u32(cl_raw);
    cl_sm = cl_raw + (((a + 1023u) & ~1023u) - a);
    if (threadIdx.x == 0) {
      tc05::mbar_init(&cl_bar[0], 1);
      tc05::mbar_init(&cl_bar[1], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // the weights arrive while the contacts are evaluated
      tc05::mbar_expect_tx(&cl_bar[0], CL_BLOB);
      tc05::bulk_g2s(cl_sm, d.clblob, CL_BLOB, &cl_bar[0]);
    }
    if (threadIdx.x < 32) {
      tc05::tmem_alloc(&cl_tmem, 64);
      tc05::tmem_relinquish();
    }
    tc05::fence_before_sync();
    __syncthreads();
    tc05::fence_after_sync();
  }
  float2 my_c = make_float2(1.0f, 1.0f);
  if (use_c && has) my_c = d.clc[cur][p];
  __shared__ int bk_s[FORCE_BLOCK_MAX / 32];
  __shared__ float bk_m[FORCE_BLOCK_MAX / 32];
  __shared__ unsigned bk_c[FORCE_BLOCK_MAX / 32];

  // ---- own sphere ----
  Owner<true> me;
  int si = 0;
  if (has) {
    si = d.sample[pc][p];
    me.pq = d.posq[cur][p];
    me.va = d.velf[cur][p];
    me.wa = d.omgf[cur][p];
    // the end of the step's per-sphere data, and the fluid cell's porosity and
    // velocity: their latency overlaps the contacts
    if (valid) {
      prefetch_l1(&d.pos[cur][p]);
      prefetch_l1(&d.vel[cur][p]);
      prefetch_l1(&d.omg[cur][p]);
      prefetch_l1(&d.posq_ref[p]);
      prefetch_l1(&d.vq[pc][p]);
      const int fc = d.fcell[pc][p];
      prefetch_l1(&d.vf[vfc][fc]);
      prefetch_l1(&d.Usf[fc]);
    }
  } else {
    me.pq = make_int4(0, 0, 0, 0);
    me.va = make_float4(0, 0, 0, 0);
    me.wa = make_float4(0, 0, 0, 0);
  }
  const SampleDev& S = d.sp[si];
  // the slot's records (the schedule's layout, k_rb_sched): entry k at rbase + k P
  const uint32_t rbase = (uint32_t)gw * (uint32_t)P * (uint32_t)d.cap + (uint32_t)sub;
  uint4* const recs = reinterpret_cast<uint4*>(d.rec[rc]);
  // the first two records are read while the list length arrives (entries
  // past a list's end, inside the warp's segment, are never dereferenced)
  uint32_t k = (uint32_t)half;
  const uint32_t cap = (uint32_t)d.cap;
  uint4 r1 = make_uint4(0u, 0u, 0u, 0u), r2 = r1;
  if (k < cap) r1 = recs[rbase + k * P];
  if (k + Lp < cap) r2 = recs[rbase + (k + Lp) * P];
  const uint32_t n = has ? d.cnt[rc][p] : 0u;
  uint32_t kmax = n;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) kmax = max(kmax, __shfl_xor_sync(FULL, kmax, o));
  V3<float> F = v3<float>(0, 0, 0), Tq = v3<float>(0, 0, 0);
  float Zacc = 0.f, Dacc = 0.f, Cacc = 0.f;  // closure data: active contacts, summed overlap, bond capacity
  // software pipeline: records are loaded two entries ahead and the next
  // entry's partner shadows one entry ahead, so neither load waits on the
  // other and both overlap the evaluation of the current entry
  int4 pq_nx = make_int4(0, 0, 0, 0);
  float4 pa_nx = make_float4(0.f, 0.f, 0.f, 0.f), pb_nx = pa_nx;
  if (k < n) {
    const uint32_t q0 = r1.x & REC_IDX;
    pq_nx = d.posq[cur][q0];
    pa_nx = d.velf[cur][q0];
    pb_nx = d.omgf[cur][q0];
  }
  for (; k < kmax; k += Lp) {
    const bool live = k < n;
    const uint4 rcur = r1;
    const int4 qq = pq_nx;
    const float4 qa = pa_nx, qb = pb_nx;
    r1 = r2;
    if (k + 2 * Lp < n) r2 = recs[rbase + (k + 2 * Lp) * P];
    if (k + Lp < n) {
      const uint32_t qn = r1.x & REC_IDX;
      pq_nx = d.posq[cur][qn];
      pa_nx = d.velf[cur][qn];
      pb_nx = d.omgf[cur][qn];
    }
    if (!live) continue;
    const size_t idx = (size_t)rbase + (size_t)k * P;
    const uint32_t pf = rcur.x;
    V3<float> xi = v3<float>(__uint_as_float(rcur.y), __uint_as_float(rcur.z), __uint_as_float(rcur.w));
    const int q = (int)(pf & REC_IDX);
    bool bonded = (pf & REC_BOND) != 0u;
    const bool had_state = (pf & (REC_BOND | REC_ACTIVE)) != 0u || xi.x != 0.f || xi.y != 0.f ||
                           xi.z != 0.f;
    bool act = false;
    if (qq.w > 0 && me.pq.w > 0) {
      const int dx = (int)((uint32_t)qq.x - (uint32_t)me.pq.x);
      const int dy = (int)((uint32_t)qq.y - (uint32_t)me.pq.y);
      const int dz = (int)((uint32_t)qq.z - (uint32_t)me.pq.z);
      const unsigned long long d2 = (unsigned long long)((long long)dx * dx) +
                                    (unsigned long long)((long long)dy * dy) +
                                    (unsigned long long)((long long)dz * dz);
      const unsigned Sq = (unsigned)me.pq.w + (unsigned)qq.w;
      const unsigned long long S2 = (unsigned long long)Sq * Sq;
      const unsigned long long band = 16ull * Sq + 256ull;
      bool touching = false, need_exact = false;
      if (d2 > S2 + band) touching = false;
      else if (d2 + band < S2) touching = true;
      else need_exact = true;
      if (bonded || touching || need_exact) {
        const float d2f = u64_to_f(d2);
        const float invd = rsqrtf(d2f);
        const float dn = d2f * invd;
        float du;
        if (d2 < (1ull << 62))
          du = __fdividef(s64_to_f((long long)S2 - (long long)d2), (float)Sq + dn);
        else
          du = (float)Sq - dn;
        const float delta = du * S.dq_f;
        const V3<float> nrm = v3<float>(dx * invd, dy * invd, dz * invd);
        const float Ri = me.va.w, Rj = qa.w, mi = me.wa.w, mj = qb.w;
        const float Rs = __fdividef(Ri * Rj, Ri + Rj);
        // surface energy of the pair: gamma sqrt(c_g,i c_g,j) under the closure
        float gam_f = S.gamma_f;
        double gam_d = S.gamma;
        const bool orig_mode = PREP && S.jkr_mode == 1;
        if (use_c && (bonded || orig_mode)) {
          const float qcg = d.clc[cur][q].y;
          gam_f = S.gamma_f * sqrtf(my_c.y * qcg);
          gam_d = S.gamma * sqrt((double)my_c.y * (double)qcg);
        }
        const bool orig = orig_mode && gam_d > 0.0;
        double d2e = 0.0, Se = 0.0;
        bool have_exact = false;
        if (need_exact) {
          exact_geometry(S, d.pos[cur][p], d.pos[cur][q], &d2e, &Se);
          have_exact = true;
          touching = d2e < __dmul_rn(Se, Se);
        }
        if (!bonded && orig && touching) bonded = true;  // original JKR: the contact forms at A
        float xs = 0.0f;  // (pi^2 gamma^2 R* / E*^2)^(1/3) of a bonded pair
        if (bonded) {
          // modified JKR: break at C for good; original JKR: separation at S
          bool broken;
          float dC = 0.0f, bandf = 4.0f * S.dq_f;
          if (gam_f > 0.f) {
            xs = m_cbrt(__fdividef(PI_F * PI_F * gam_f * gam_f * Rs, S.Es_f * S.Es_f));
            dC = (orig ? -1.1905507889761495f : -0.57235712127666594f) * xs;
            bandf += 2e-5f * fabsf(dC);
          }
          if (delta < dC - bandf) {
            broken = true;
          } else if (delta > dC + bandf) {
            broken = false;
          } else {
            const double4 A = d.pos[cur][p], B = d.pos[cur][q];
            if (!have_exact) {
              exact_geometry(S, A, B, &d2e, &Se);
              have_exact = true;
              touching = d2e < __dmul_rn(Se, Se);
            }
            const double Rid = fabs(A.w), Rjd = fabs(B.w);
            const double Rsd = __dmul_rn(Rid, Rjd) / __dadd_rn(Rid, Rjd);
            const double de = __dsub_rn(Se, sqrt(d2e));
            broken = orig ? contact_separates_exact(de, Rsd, S.Es, gam_d) : bond_breaks_exact(de, Rsd, S.Es, gam_d);
          }
          if (broken) bonded = false;
        }
        act = bonded || touching;
        if (act) {
          const float ms = __fdividef(mi * mj, mi + mj);
          const V3<float> vrel = v3<float>(qa.x - me.va.x, qa.y - me.va.y, qa.z - me.va.z);
          const V3<float> rw = v3<float>(Ri * me.wa.x + Rj * qb.x, Ri * me.wa.y + Rj * qb.y,
                                         Ri * me.wa.z + Rj * qb.z);
          const V3<float> rwn = cross3(rw, nrm);
          const V3<float> vc = v3<float>(vrel.x - rwn.x, vrel.y - rwn.y, vrel.z - rwn.z);
          V3<float> Fi, Ft;
          contact_law_mixed(delta, nrm, vrel, vc, Rs, ms, gam_f, bonded, 2.5198420997897464f * xs, S, xi,
                            Fi, Ft, orig);  // d_A = 16^(1/3) xs
          const V3<float> nFt = cross3(nrm, Ft);
          F.x += Fi.x;
          F.y += Fi.y;
          F.z += Fi.z;
          Tq.x += Ri * nFt.x;
          Tq.y += Ri * nFt.y;
          Tq.z += Ri * nFt.z;
          if (feat) {
            Zacc += 1.f;
            Dacc += delta;
            Cacc += bonded ? 0.5f * 3.0f * PI_F * gam_f * Rs : 0.0f;
          }
        }
      }
    }
    // write the record back when its state changed
    if (act) {
      const uint32_t npf = (uint32_t)q | REC_ACTIVE | (bonded ? REC_BOND : 0u);
      recs[idx] = make_uint4(npf, __float_as_uint(xi.x), __float_as_uint(xi.y), __float_as_uint(xi.z));
    } else if (had_state) {
      recs[idx] = make_uint4((uint32_t)q, 0u, 0u, 0u);
    }
  }
  if (Lp == 2) {  // two lanes per sphere: the odd entries' sums join the even ones'
    F.x += __shfl_down_sync(FULL, F.x, 16);
    F.y += __shfl_down_sync(FULL, F.y, 16);
    F.z += __shfl_down_sync(FULL, F.z, 16);
    Tq.x += __shfl_down_sync(FULL, Tq.x, 16);
    Tq.y += __shfl_down_sync(FULL, Tq.y, 16);
    Tq.z += __shfl_down_sync(FULL, Tq.z, 16);
    if (feat) {
      Zacc += __shfl_down_sync(FULL, Zacc, 16);
      Dacc += __shfl_down_sync(FULL, Dacc, 16);
      Cacc += __shfl_down_sync(FULL, Cacc, 16);
    }
  }
  finish_step<true, MODE, CL, PREP>(d, ctl, cur, nxt, pc, vfc, m_step, couple_next, epoch, lane, valid, p, si, me,
                              F, Tq, Zacc, Dacc, Cacc, my_c, use_c, feat, rec, net, cl_sm, cl_bar, cl_tmem,
                              &bk_n, bk_s, bk_m, bk_c, h_next, h_fluid);
}


// MODE_CANON bookkeeping kernel (single thread).
__global__ void k_after_canon(Dev d) {
  Ctl* ctl = d.ctl;
  ctl->cur ^= 1;
  ctl->step += 1;
}

void launch_forces(const Dev& d, int mode, int block, cudaStream_t s, cudaGraphConditionalHandle h_next,
    cudaGraphConditionalHandle h_fluid) {
  // Npad is a multiple of 256, so every block size divides it exactly
  // (a context with the learned closure runs blocks of 128: one M = 128 tile)
  // The closure variant only while the closure is on or recording: its
  // tiles' shared memory shrinks the L1 cache the neighbour gathers hit,
  // and its registers the occupancy.  With both off the plain kernel
  // computes the same step (corrections 1).
  const bool cl = d.clblob && (d.cl_smem || d.cl_rec);
  const int B = cl ? 128 : ((block == 64 || block == 256) ? block : 128);
  const int grid = d.Npad * (32 / d.ppw) / B;
  const size_t sm = (cl && d.cl_smem) ? CL_SMEM : 0;
  if (d.N == 0) return;
  // PREP: the kernels that also run the preparation stages (original JKR,
  // moving plate and penetrometer), once a context has used them
  if (cl) {
    if (d.mixed) {
      if (mode == MODE_FORCES) k_forces_lanes<MODE_FORCES, true, false><<<grid, B, sm, s>>>(d, 0, 0);
      else if (mode == MODE_MID) k_forces_lanes<MODE_MID, true, false><<<grid, B, sm, s>>>(d, h_next, h_fluid);
      else k_forces_lanes<MODE_CANON, true, false><<<grid, B, sm, s>>>(d, 0, 0);
    } else {
      if (mode == MODE_FORCES) k_forces_pairs<MODE_FORCES, true, false><<<grid, B, sm, s>>>(d, 0, 0);
      else if (mode == MODE_MID) k_forces_pairs<MODE_MID, true, false><<<grid, B, sm, s>>>(d, h_next, h_fluid);
      else k_forces_pairs<MODE_CANON, true, false><<<grid, B, sm, s>>>(d, 0, 0);
    }
  } else if (d.mixed && d.prep) {
    if (mode == MODE_FORCES) k_forces_lanes<MODE_FORCES, false, true><<<grid, B, 0, s>>>(d, 0, 0);
    else if (mode == MODE_MID) k_forces_lanes<MODE_MID, false, true><<<grid, B, 0, s>>>(d, h_next, h_fluid);
    else k_forces_lanes<MODE_CANON, false, true><<<grid, B, 0, s>>>(d, 0, 0);
  } else if (d.mixed) {
    if (mode == MODE_FORCES) k_forces_lanes<MODE_FORCES, false, false><<<grid, B, 0, s>>>(d, 0, 0);
    else if (mode == MODE_MID) k_forces_lanes<MODE_MID, false, false><<<grid, B, 0, s>>>(d, h_next, h_fluid);
    else k_forces_lanes<MODE_CANON, false, false><<<grid, B, 0, s>>>(d, 0, 0);
  } else if (d.prep) {
    if (mode == MODE_FORCES) k_forces_pairs<MODE_FORCES, false, true><<<grid, B, 0, s>>>(d, 0, 0);
    else if (mode == MODE_MID) k_forces_pairs<MODE_MID, false, true><<<grid, B, 0, s>>>(d, h_next, h_fluid);
    else k_forces_pairs<MODE_CANON, false, true><<<grid, B, 0, s>>>(d, 0, 0);
  } else {
    if (mode == MODE_FORCES) k_forces_pairs<MODE_FORCES, false, false><<<grid, B, 0, s>>>(d, 0, 0);
    else if (mode == MODE_MID) k_forces_pairs<MODE_MID, false, false><<<grid, B, 0, s>>>(d, h_next, h_fluid);
    else k_forces_pairs<MODE_CANON, false, false><<<grid, B, 0, s>>>(d, 0, 0);
  }
  if (mode == MODE_CANON) k_after_canon<<<1, 1, 0, s>>>(d);
}

}  // namespace cgdem
