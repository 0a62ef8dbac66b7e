// k_forces.cu -- contact, wall, body and drag forces of one DEM step fused
// with the velocity-Verlet update (arXiv 2211.06142, Sec. 2.1-2.3).
//
// One thread per particle walks its candidate list (ELL, column-major) and
// sums its own contacts in list order; every pair is evaluated from both
// sides with bit-identical magnitudes, so no float atomics are needed and
// the result is deterministic.
//
// Two precisions:
//   FP64  -- geometry and contact physics in double.
//   MIXED -- positions, integrator and accumulators stay FP64, the contact
//            geometry comes from a per-step 32-bit fixed-point shadow of the
//            positions (exact integer differences, so the overlap
//            delta = Ri + Rj - d suffers no cancellation), and the contact
//            physics and tangential history run in FP32.  Every integer
//            decision (touching, bond break) is taken in IEEE double from the
//            FP64 positions whenever the fixed-point value lies within its
//            error band of the threshold, so it always equals the FP64
//            decision.  GB300 runs FP64 at ~1/60 of the FP32 rate, so the
//            common path holds no FP64 arithmetic per contact.
#include "cgdem_internal.cuh"

namespace cgdem {

constexpr double PI_D = 3.14159265358979323846;
constexpr float PI_F = 3.14159265358979323846f;

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
  static constexpr int newton_iters = 6;
};

// Contact radius and elastic normal force on the stable JKR branch
// (Eq. 12-13), solved in reduced units: with a_A^3 = 4 pi gamma R*^2 / E*
// (Table 1, point A) and u^2 = a / a_A, Eq. 13 reads u^4 - u = delta / d_A
// with d_A = a_A^2 / R*, and Eq. 12 reads F = pi gamma R* (16/3 u^6 - 8 u^3).
// Newton from above converges monotonically (the quartic is convex and
// increasing for u > 4^(-1/3); the stable branch starts at u_C = (3/4)^(1/3)).
template <typename T>
__device__ __forceinline__ void jkr_solve(T delta, T Rs, T Es, T gamma, T* a_out, T* F_out) {
  const T pi = Consts<T>::pi();
  T aA = cbrtT(T(4) * pi * gamma * Rs * Rs / Es);
  T dA = aA * aA / Rs;
  T D = delta / dA;
  T u = D >= T(0) ? sqrtT(sqrtT(D + T(1))) + T(0.05) : T(1);
#pragma unroll
  for (int it = 0; it < Consts<T>::newton_iters; ++it) {
    T u3 = u * u * u;
    u -= (u3 * u - u - D) / (T(4) * u3 - T(1));
  }
  const T uC = T(0.90856029641606983);  // (3/4)^(1/3)
  if (u < uC) u = uC;
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
                                            int coulomb_mode, V3<T>& xi, V3<T>& Fi, V3<T>& Ft) {
  T a, Fne;
  if (bonded && gamma > T(0)) {
    jkr_solve<T>(delta, Rs, Es, gamma, &a, &Fne);
  } else {
    a = delta > T(0) ? sqrtT(Rs * delta) : T(0);
    Fne = T(4) * Es * a * a * a / (T(3) * Rs);
  }
  const T cd = Consts<T>::damp();
  T gn = cd * beta * sqrtT(T(2) * Es * a * ms);  // Eq. 32
  T vn = dot3(vrel, n);
  T Fn = Fne - gn * vn;
  // tangential spring rotated into the tangent plane, Eq. 4
  T vcn = dot3(vc, n);
  V3<T> vt = v3<T>(vc.x - vcn * n.x, vc.y - vcn * n.y, vc.z - vcn * n.z);
  T old = sqrtT(dot3(xi, xi));
  T xn = dot3(xi, n);
  xi.x -= xn * n.x;
  xi.y -= xn * n.y;
  xi.z -= xn * n.z;
  T nw = sqrtT(dot3(xi, xi));
  if (nw > T(0)) {
    T sc = old / nw;
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
  T gt = cd * beta * sqrtT(kt * ms);
  Ft = v3<T>(kt * xi.x + gt * vt.x, kt * xi.y + gt * vt.y, kt * xi.z + gt * vt.z);
  T FC = T(3) * Consts<T>::pi() * gamma * Rs;  // Table 1
  T Flim = coulomb_mode == 1 ? fabs(Fne) : (bonded ? Fne + T(2) * FC : Fne);
  if (Flim < T(0)) Flim = T(0);
  T ftm = sqrtT(dot3(Ft, Ft));
  T cap = mu * Flim;  // Eq. 35
  if (ftm > cap) {
    T sc = ftm > T(0) ? cap / ftm : T(0);
    Ft.x *= sc;
    Ft.y *= sc;
    Ft.z *= sc;
    if (kt > T(0)) {
      xi.x = (Ft.x - gt * vt.x) / kt;
      xi.y = (Ft.y - gt * vt.y) / kt;
      xi.z = (Ft.z - gt * vt.z) / kt;
    }
  }
  Fi = v3<T>(-Fn * n.x + Ft.x, -Fn * n.y + Ft.y, -Fn * n.z + Ft.z);
}

// Di Felice drag (Eq. 8-11) written as (pi d^2 / 8) (0.63 sqrt(rho_f |w|)
// + 4.8 sqrt(mu_f / d))^2 w n^-chi, which equals Eq. 8 with Eq. 9 and stays
// finite as Re -> 0.
template <typename T>
__device__ __forceinline__ V3<T> drag_force(T rho_f, T mu_f, T dp, V3<T> w, T n) {
  T wm = sqrtT(dot3(w, w));
  if (!(wm > T(0))) return v3<T>(0, 0, 0);
  T Re = rho_f * dp * wm / mu_f;
  T lr = T(1.5) - log10T(Re);
  T chi = T(3.7) - T(0.65) * expT(-(lr * lr) * T(0.5));
  T t = T(0.63) * sqrtT(rho_f * wm) + T(4.8) * sqrtT(mu_f / dp);
  T pre = Consts<T>::pi() * dp * dp / T(8) * t * t * powT(n, -chi);
  return v3<T>(pre * w.x, pre * w.y, pre * w.z);
}

__device__ __forceinline__ float ll2f(long long v) { return __ll2float_rn(v); }
__device__ __forceinline__ float ull2f(unsigned long long v) { return __ull2float_rn(v); }

enum { MODE_FORCES = 0, MODE_MID = 1, MODE_CANON = 2 };

// Per-sample atomic maximum of a non-negative double (as ordered bits).
__device__ __forceinline__ void atomic_max_pos(unsigned long long* addr, double v) {
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// Wall contacts of the cylinder (Sec. 3.1: Hertz particle-wall law).
template <typename T>
__device__ __forceinline__ void wall_contacts(const SampleDev& s, double4 P, V3<T> v, V3<T> w,
                                              T R, T m, T Es, T Gs, T beta, T mu, T dt,
                                              V3<T>* hist, V3<T>& F, V3<T>& Tq, bool* changed) {
  const double r2 = __dadd_rn(__dmul_rn(P.x, P.x), __dmul_rn(P.y, P.y));
  for (int wall = 0; wall < 3; ++wall) {
    double delta = -1.0;
    V3<T> n = v3<T>(0, 0, 0);
    if (wall == 0) {
      double lim = s.Rc - fabs(P.w);
      if (lim < 0) lim = 0;
      if (r2 > lim * lim * (1.0 - 1e-6) && r2 > 0.0) {
        double r = sqrt(r2);
        delta = (r + fabs(P.w)) - s.Rc;
        n = v3<T>(T(P.x / r), T(P.y / r), T(0));
      }
    } else if (wall == 1) {
      if (P.z < fabs(P.w) && sqrt(r2) >= s.r_out) {
        delta = fabs(P.w) - P.z;
        n = v3<T>(0, 0, -1);
      }
    } else {
      delta = (P.z + fabs(P.w)) - s.H;
      n = v3<T>(0, 0, 1);
    }
    if (!(delta > 0.0)) {
      if (hist[wall].x != T(0) || hist[wall].y != T(0) || hist[wall].z != T(0)) {
        hist[wall] = v3<T>(0, 0, 0);
        changed[wall] = true;
      }
      continue;
    }
    V3<T> vrel = v3<T>(-v.x, -v.y, -v.z);
    V3<T> rw = v3<T>(R * w.x, R * w.y, R * w.z);
    V3<T> rwn = cross3(rw, n);
    V3<T> vc = v3<T>(vrel.x - rwn.x, vrel.y - rwn.y, vrel.z - rwn.z);
    V3<T> Fi, Ft;
    contact_law<T>(T(delta), n, vrel, vc, R, m, T(0), false, Es, Gs, beta, mu, dt, s.coulomb_mode,
                   hist[wall], Fi, Ft);
    changed[wall] = true;
    V3<T> nFt = cross3(n, Ft);
    F.x += Fi.x;
    F.y += Fi.y;
    F.z += Fi.z;
    Tq.x += R * nFt.x;
    Tq.y += R * nFt.y;
    Tq.z += R * nFt.z;
  }
}

template <bool MIXED, int MODE>
__global__ void __launch_bounds__(256) k_forces(Dev d) {
  using T = typename std::conditional<MIXED, float, double>::type;
  Ctl* ctl = d.ctl;
  const int cur = ctl->cur;
  const int nxt = cur ^ 1;
  const int pc = ctl->pcur;
  const int rc = ctl->rec_cur;
  const int vfc = ctl->vf_cur;
  const long long m_step = ctl->step + 1;  // step completed by this evaluation
  const int Npad = d.Npad;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;

  __shared__ int s_uniform_sample;
  __shared__ unsigned long long s_vmax;
  __shared__ int s_couple_any;
  if (threadIdx.x == 0) {
    s_uniform_sample = -2;
    s_vmax = 0ull;
    s_couple_any = 0;
  }
  __syncthreads();

  int my_sample = -1;
  double my_disp2 = -1.0;
  bool coupled = false;

  if (p < d.N) {
    double4 P = d.pos[cur][p];
    double4 Vd = d.vel[cur][p];
    double4 Wd = d.omg[cur][p];
    const int si = d.sample[pc][p];
    my_sample = si;
    const SampleDev& S = d.sp[si];
    const bool active = P.w > 0.0;
    if (!active) {
      if (MODE != MODE_FORCES) {
        d.pos[nxt][p] = P;
        d.vel[nxt][p] = Vd;
        d.omg[nxt][p] = Wd;
        d.posq[nxt][p] = d.posq[cur][p];
        d.velf[nxt][p] = d.velf[cur][p];
        d.omgf[nxt][p] = d.omgf[cur][p];
      }
      if (MODE != MODE_MID) {
        d.F[p] = make_double4(0, 0, 0, 0);
        d.T[p] = make_double4(0, 0, 0, 0);
      }
    } else {
      const T Es = T(S.Es), Gs = T(S.Gs), beta = T(S.beta), mu = T(S.mu), gam = T(S.gamma);
      const T dt = T(S.dt);
      V3<T> F = v3<T>(0, 0, 0), Tq = v3<T>(0, 0, 0);
      // own particle in working precision
      T Ri, mi;
      V3<T> vi, wi;
      int4 pq;
      if (MIXED) {
        pq = d.posq[cur][p];
        float4 a = d.velf[cur][p];
        float4 b = d.omgf[cur][p];
        vi = v3<T>(a.x, a.y, a.z);
        Ri = a.w;
        wi = v3<T>(b.x, b.y, b.z);
        mi = b.w;
      } else {
        vi = v3<T>(Vd.x, Vd.y, Vd.z);
        wi = v3<T>(Wd.x, Wd.y, Wd.z);
        Ri = P.w;
        mi = 1.0 / Vd.w;
      }
      const uint32_t ncand = d.cnt[rc][p];
      for (uint32_t k = 0; k < ncand; ++k) {
        const size_t idx = (size_t)k * Npad + p;
        uint32_t pf;
        V3<T> xi;
        if (MIXED) {
          uint4 r = reinterpret_cast<const uint4*>(d.rec[rc])[idx];
          pf = r.x;
          xi = v3<T>(__uint_as_float(r.y), __uint_as_float(r.z), __uint_as_float(r.w));
        } else {
          const RecD* rr = reinterpret_cast<const RecD*>(d.rec[rc]) + idx;
          int4 h0 = *reinterpret_cast<const int4*>(rr);
          double2 h1 = *(reinterpret_cast<const double2*>(rr) + 1);
          pf = (uint32_t)h0.x;
          xi = v3<T>(__hiloint2double(h0.w, h0.z), h1.x, h1.y);
        }
        const int q = (int)(pf & REC_IDX);
        bool bonded = (pf & REC_BOND) != 0u;
        const bool had_state = (pf & (REC_BOND | REC_ACTIVE)) != 0u || xi.x != T(0) ||
                               xi.y != T(0) || xi.z != T(0);
        bool touching = false, act = false;
        T delta = 0, Rj = 0, mj = 0;
        V3<T> n = v3<T>(0, 0, 0), vj = v3<T>(0, 0, 0), wj = v3<T>(0, 0, 0);
        double4 Q;
        bool q_active;
        if (MIXED) {
          int4 qq = d.posq[cur][q];
          q_active = qq.w > 0;
          if (q_active) {
            const int dx = (int)((uint32_t)qq.x - (uint32_t)pq.x);
            const int dy = (int)((uint32_t)qq.y - (uint32_t)pq.y);
            const int dz = (int)((uint32_t)qq.z - (uint32_t)pq.z);
            const unsigned long long d2 = (unsigned long long)((long long)dx * dx) +
                                          (unsigned long long)((long long)dy * dy) +
                                          (unsigned long long)((long long)dz * dz);
            const unsigned Sq = (unsigned)pq.w + (unsigned)qq.w;
            const unsigned long long S2 = (unsigned long long)Sq * Sq;
            const unsigned long long band = 16ull * Sq + 256ull;
            bool need_exact = false;
            if (d2 > S2 + band) {
              touching = false;
            } else if (d2 + band < S2) {
              touching = true;
            } else {
              need_exact = true;
            }
            if (!bonded && !touching && !need_exact) {
              act = false;
            } else {
              const float dn = sqrtf(ull2f(d2));
              float du;
              if (d2 < (1ull << 62))
                du = ll2f((long long)S2 - (long long)d2) / ((float)Sq + dn);
              else
                du = (float)Sq - dn;
              delta = du * S.dq_f;
              const float invd = 1.0f / dn;
              n = v3<T>(dx * invd, dy * invd, dz * invd);
              float4 qa = d.velf[cur][q];
              float4 qb = d.omgf[cur][q];
              vj = v3<T>(qa.x, qa.y, qa.z);
              Rj = qa.w;
              wj = v3<T>(qb.x, qb.y, qb.z);
              mj = qb.w;
              const T Rs = Ri * Rj / (Ri + Rj);
              double d2e = 0.0, Se = 0.0;
              bool have_exact = false;
              if (need_exact) {
                exact_geometry(S, P, d.pos[cur][q], &d2e, &Se);
                have_exact = true;
                touching = d2e < __dmul_rn(Se, Se);
              }
              if (bonded) {
                bool broken;
                float dC = 0.0f, bandf;
                if (gam > T(0)) {
                  float xs = cbrtf(PI_F * PI_F * gam * gam * Rs / (Es * Es));
                  dC = -0.57235712127666594f * xs;
                  bandf = 4.0f * S.dq_f + 2e-5f * fabsf(dC);
                } else {
                  bandf = 4.0f * S.dq_f;
                }
                if (delta < dC - bandf) {
                  broken = true;
                } else if (delta > dC + bandf) {
                  broken = false;
                } else {
                  if (!have_exact) {
                    exact_geometry(S, P, d.pos[cur][q], &d2e, &Se);
                    have_exact = true;
                    touching = d2e < __dmul_rn(Se, Se);
                  }
                  const double Rid = fabs(P.w), Rjd = fabs(d.pos[cur][q].w);
                  const double Rsd = __dmul_rn(Rid, Rjd) / __dadd_rn(Rid, Rjd);
                  broken = bond_breaks_exact(__dsub_rn(Se, sqrt(d2e)), Rsd, S.Es, S.gamma);
                }
                if (broken) bonded = false;
              }
              act = bonded || touching;
              if (act) {
                const T ms = mi * mj / (mi + mj);
                V3<T> vrel = v3<T>(vj.x - vi.x, vj.y - vi.y, vj.z - vi.z);
                V3<T> rw = v3<T>(Ri * wi.x + Rj * wj.x, Ri * wi.y + Rj * wj.y, Ri * wi.z + Rj * wj.z);
                V3<T> rwn = cross3(rw, n);
                V3<T> vc = v3<T>(vrel.x - rwn.x, vrel.y - rwn.y, vrel.z - rwn.z);
                V3<T> Fi, Ft;
                contact_law<T>(delta, n, vrel, vc, Rs, ms, gam, bonded, Es, Gs, beta, mu, dt,
                               S.coulomb_mode, xi, Fi, Ft);
                V3<T> nFt = cross3(n, Ft);
                F.x += Fi.x;
                F.y += Fi.y;
                F.z += Fi.z;
                Tq.x += Ri * nFt.x;
                Tq.y += Ri * nFt.y;
                Tq.z += Ri * nFt.z;
              }
            }
          }
        } else {
          Q = d.pos[cur][q];
          q_active = Q.w > 0.0;
          if (q_active) {
            double dx = __dsub_rn(Q.x, P.x), dy = __dsub_rn(Q.y, P.y), dz = __dsub_rn(Q.z, P.z);
            if (S.kind == CGDEM_PERIODIC_BOX) {
              dx = min_image(dx, S.L[0]);
              dy = min_image(dy, S.L[1]);
              dz = min_image(dz, S.L[2]);
            }
            const double d2 =
                __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            const double Sd = __dadd_rn(P.w, Q.w);
            touching = d2 < __dmul_rn(Sd, Sd);
            if (bonded || touching) {
              const double dist = sqrt(d2);
              const double Rs = __dmul_rn(P.w, Q.w) / __dadd_rn(P.w, Q.w);
              delta = __dsub_rn(Sd, dist);
              if (bonded && bond_breaks_exact(delta, Rs, S.Es, S.gamma)) bonded = false;
              act = bonded || touching;
              if (act && dist > 0.0) {
                double4 QV = d.vel[cur][q];
                double4 QW = d.omg[cur][q];
                Rj = Q.w;
                mj = 1.0 / QV.w;
                n = v3<T>(dx / dist, dy / dist, dz / dist);
                vj = v3<T>(QV.x, QV.y, QV.z);
                wj = v3<T>(QW.x, QW.y, QW.z);
                const T ms = mi * mj / (mi + mj);
                V3<T> vrel = v3<T>(vj.x - vi.x, vj.y - vi.y, vj.z - vi.z);
                V3<T> rw = v3<T>(Ri * wi.x + Rj * wj.x, Ri * wi.y + Rj * wj.y, Ri * wi.z + Rj * wj.z);
                V3<T> rwn = cross3(rw, n);
                V3<T> vc = v3<T>(vrel.x - rwn.x, vrel.y - rwn.y, vrel.z - rwn.z);
                V3<T> Fi, Ft;
                contact_law<T>(delta, n, vrel, vc, Rs, ms, gam, bonded, Es, Gs, beta, mu, dt,
                               S.coulomb_mode, xi, Fi, Ft);
                V3<T> nFt = cross3(n, Ft);
                F.x += Fi.x;
                F.y += Fi.y;
                F.z += Fi.z;
                Tq.x += Ri * nFt.x;
                Tq.y += Ri * nFt.y;
                Tq.z += Ri * nFt.z;
              } else if (act) {
                act = false;  // coincident centres: no normal defined
              }
            }
          }
        }
        // write the record back when its state changed
        if (act) {
          uint32_t npf = (uint32_t)q | REC_ACTIVE | (bonded ? REC_BOND : 0u);
          if (MIXED) {
            reinterpret_cast<uint4*>(d.rec[rc])[idx] =
                make_uint4(npf, __float_as_uint((float)xi.x), __float_as_uint((float)xi.y),
                           __float_as_uint((float)xi.z));
          } else {
            RecD* rr = reinterpret_cast<RecD*>(d.rec[rc]) + idx;
            double xx = (double)xi.x;
            *reinterpret_cast<int4*>(rr) =
                make_int4((int)npf, 0, __double2loint(xx), __double2hiint(xx));
            *(reinterpret_cast<double2*>(rr) + 1) = make_double2((double)xi.y, (double)xi.z);
          }
        } else if (had_state) {
          if (MIXED) {
            reinterpret_cast<uint4*>(d.rec[rc])[idx] = make_uint4((uint32_t)q, 0u, 0u, 0u);
          } else {
            RecD* rr = reinterpret_cast<RecD*>(d.rec[rc]) + idx;
            *reinterpret_cast<int4*>(rr) = make_int4(q, 0, 0, 0);
            *(reinterpret_cast<double2*>(rr) + 1) = make_double2(0.0, 0.0);
          }
        }
      }

      // walls of the cylindrical sample
      if (S.kind == CGDEM_CYLINDER) {
        V3<T> hist[3];
        bool changed[3] = {false, false, false};
        if (MIXED) {
#pragma unroll
          for (int w = 0; w < 3; ++w) {
            float4 h = d.wallhf[pc][(size_t)w * Npad + p];
            hist[w] = v3<T>(h.x, h.y, h.z);
          }
        } else {
#pragma unroll
          for (int w = 0; w < 3; ++w) {
            double4 h = d.wallh[pc][(size_t)w * Npad + p];
            hist[w] = v3<T>(h.x, h.y, h.z);
          }
        }
        wall_contacts<T>(S, P, vi, wi, Ri, mi, Es, Gs, beta, mu, dt, hist, F, Tq, changed);
#pragma unroll
        for (int w = 0; w < 3; ++w) {
          if (!changed[w]) continue;
          if (MIXED)
            d.wallhf[pc][(size_t)w * Npad + p] =
                make_float4((float)hist[w].x, (float)hist[w].y, (float)hist[w].z, 0.f);
          else
            d.wallh[pc][(size_t)w * Npad + p] =
                make_double4((double)hist[w].x, (double)hist[w].y, (double)hist[w].z, 0.0);
        }
      }

      // gravity, buoyancy (Eq. 1) and drag (Eq. 8-11)
      {
        const T rho_s = T(S.rho);
        const T Vp = mi / rho_s;
        const T rf = T(S.rho_f);
        F.x += mi * T(S.g[0]);
        F.y += mi * T(S.g[1]);
        F.z += mi * T(S.g[2]);
        if (S.use_buoyancy) {
          F.x -= rf * Vp * T(S.g[0]);
          F.y -= rf * Vp * T(S.g[1]);
          F.z -= rf * Vp * T(S.g[2]);
        }
        if (S.use_drag) {
          const int fc = d.fcell[pc][p];
          const unsigned long long Sc = d.vf[vfc][fc];
          T nc = T(1) - (MIXED ? T(ull2f(Sc)) : T((double)Sc)) * T(9.094947017729282379150390625e-13);
          if (nc < T(S.n_min)) nc = T(S.n_min);
          if (nc > T(1)) nc = T(1);
          V3<T> U;
          if (MIXED) {
            float4 u = d.Usf[fc];
            U = v3<T>(u.x, u.y, u.z);
          } else {
            double4 u = d.Us[fc];
            U = v3<T>(u.x, u.y, u.z);
          }
          V3<T> w = v3<T>(U.x / nc - vi.x, U.y / nc - vi.y, U.z / nc - vi.z);
          V3<T> fd = drag_force<T>(rf, T(S.mu_f), T(2) * Ri, w, nc);
          F.x += fd.x;
          F.y += fd.y;
          F.z += fd.z;
        }
      }

      const double Fx = (double)F.x, Fy = (double)F.y, Fz = (double)F.z;
      const double Tx = (double)Tq.x, Ty = (double)Tq.y, Tz = (double)Tq.z;
      if (!isfinite(Fx + Fy + Fz + Tx + Ty + Tz)) latch(ctl, ST_NONFINITE);

      if (MODE == MODE_FORCES) {
        d.F[p] = make_double4(Fx, Fy, Fz, 0.0);
        d.T[p] = make_double4(Tx, Ty, Tz, 0.0);
      } else {
        // velocity Verlet: complete this step's kick, then (MODE_MID) the
        // next step's half kick and drift.
        const double h = S.half_dt;
        const double im = Vd.w, iI = Wd.w;
        double vx, vy, vz, wx, wy, wz;
        bool removed = false;
        if (MODE == MODE_CANON || !MIXED) {
          vx = Vd.x + h * (Fx * im);
          vy = Vd.y + h * (Fy * im);
          vz = Vd.z + h * (Fz * im);
          wx = Wd.x + h * (Tx * iI);
          wy = Wd.y + h * (Ty * iI);
          wz = Wd.z + h * (Tz * iI);
        }
        if (S.kind == CGDEM_CYLINDER && P.z < -2.0 * P.w) {  // outlet (Eq. 40 produced sand)
          removed = true;
          d.removed_step[d.id[pc][p]] = (int)m_step;
        }
        if (MODE == MODE_CANON) {
          d.F[p] = make_double4(Fx, Fy, Fz, 0.0);
          d.T[p] = make_double4(Tx, Ty, Tz, 0.0);
          double4 Pn = P;
          if (removed) Pn.w = -P.w;
          d.pos[nxt][p] = Pn;
          d.vel[nxt][p] = make_double4(vx, vy, vz, Vd.w);
          d.omg[nxt][p] = make_double4(wx, wy, wz, Wd.w);
          int4 pqn = d.posq[cur][p];
          if (removed) pqn.w = 0;
          d.posq[nxt][p] = pqn;
          d.velf[nxt][p] = make_float4((float)vx, (float)vy, (float)vz, (float)P.w);
          d.omgf[nxt][p] = make_float4((float)wx, (float)wy, (float)wz, (float)(1.0 / Vd.w));
        } else {
          if (MIXED) {
            // both half kicks at once: v(n+1/2) = v(n-1/2) + dt F / m
            const double c = S.dt * im, cI = S.dt * iI;
            vx = Vd.x + c * Fx;
            vy = Vd.y + c * Fy;
            vz = Vd.z + c * Fz;
            wx = Wd.x + cI * Tx;
            wy = Wd.y + cI * Ty;
            wz = Wd.z + cI * Tz;
          } else {
            vx += h * (Fx * im);
            vy += h * (Fy * im);
            vz += h * (Fz * im);
            wx += h * (Tx * iI);
            wy += h * (Ty * iI);
            wz += h * (Tz * iI);
          }
          if (removed) {
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
            if (S.kind == CGDEM_PERIODIC_BOX) {
              if (x >= S.L[0]) x -= S.L[0]; else if (x < 0.0) x += S.L[0];
              if (y >= S.L[1]) y -= S.L[1]; else if (y < 0.0) y += S.L[1];
              if (z >= S.L[2]) z -= S.L[2]; else if (z < 0.0) z += S.L[2];
            }
            d.pos[nxt][p] = make_double4(x, y, z, P.w);
            d.vel[nxt][p] = make_double4(vx, vy, vz, Vd.w);
            d.omg[nxt][p] = make_double4(wx, wy, wz, Wd.w);
            int4 pqn = d.posq[cur][p];
            pqn.x = to_q(x, S.inv_dq);
            pqn.y = to_q(y, S.inv_dq);
            pqn.z = to_q(z, S.inv_dq);
            d.posq[nxt][p] = pqn;
            d.velf[nxt][p] = make_float4((float)vx, (float)vy, (float)vz, (float)P.w);
            d.omgf[nxt][p] = make_float4((float)wx, (float)wy, (float)wz, (float)(1.0 / Vd.w));
            const double ddx = S.dt * vx, ddy = S.dt * vy, ddz = S.dt * vz;
            my_disp2 = ddx * ddx + ddy * ddy + ddz * ddz;
            const int fc = fluid_cell_of(S, x, y, z);
            d.fcell[pc][p] = fc;
            if (m_step % S.couple_every == 0) {
              coupled = true;
              if (S.vf_mode == 0) {
                atomicAdd(&d.vf[(vfc + 1) % 3][fc], d.vq[pc][p]);
              }
            }
          }
        }
      }
    }
  }

  if (MODE != MODE_MID) return;

  // ---- per-sample displacement bound, porosity rotation, step bookkeeping
  // zero the porosity buffer that the step after next will fill
  {
    unsigned long long* z = d.vf[(vfc + 2) % 3];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < d.Cf_total; c += gridDim.x * blockDim.x)
      z[c] = 0ull;
  }
  if (coupled) s_couple_any = 1;
  // block-uniform sample: one atomic per block
  if (my_sample >= 0) atomicCAS(&s_uniform_sample, -2, my_sample);
  __syncthreads();
  const int us = s_uniform_sample;
  bool uniform = __syncthreads_and(my_sample < 0 || my_sample == us);
  if (my_disp2 >= 0.0) {
    if (uniform)
      atomicMax(&s_vmax, (unsigned long long)__double_as_longlong(my_disp2));
    else
      atomic_max_pos(&d.vmax2[my_sample], my_disp2);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (uniform && us >= 0 && s_vmax != 0ull) atomicMax(&d.vmax2[us], s_vmax);
    if (s_couple_any) atomicOr(&ctl->coupled, 1u);
    __threadfence();
    unsigned t = atomicAdd(&ctl->block_counter, 1u);
    if (t == gridDim.x - 1) {
      __threadfence();
      for (int s = 0; s < d.n_samples; ++s) {
        unsigned long long b = atomicExch(&d.vmax2[s], 0ull);
        double dd = d.disp[s] + sqrt(__longlong_as_double((long long)b));
        d.disp[s] = dd;
        if (2.0 * dd > d.sp[s].rebuild_disp) ctl->rebuild = 1;
      }
      if (atomicExch(&ctl->coupled, 0u)) ctl->vf_cur = (vfc + 1) % 3;
      ctl->cur = nxt;
      ctl->step = m_step;
      ctl->block_counter = 0u;
      __threadfence();
    }
  }
}

// MODE_CANON / MODE_FORCES bookkeeping kernel (single thread).
__global__ void k_after_canon(Dev d) {
  Ctl* ctl = d.ctl;
  ctl->cur ^= 1;
  ctl->step += 1;
}

void launch_forces(const Dev& d, int mode, int block, cudaStream_t s) {
  const int grid = (d.N + block - 1) / block;
  if (grid == 0) return;
  if (d.mixed) {
    if (mode == MODE_FORCES) k_forces<true, MODE_FORCES><<<grid, block, 0, s>>>(d);
    else if (mode == MODE_MID) k_forces<true, MODE_MID><<<grid, block, 0, s>>>(d);
    else k_forces<true, MODE_CANON><<<grid, block, 0, s>>>(d);
  } else {
    if (mode == MODE_FORCES) k_forces<false, MODE_FORCES><<<grid, block, 0, s>>>(d);
    else if (mode == MODE_MID) k_forces<false, MODE_MID><<<grid, block, 0, s>>>(d);
    else k_forces<false, MODE_CANON><<<grid, block, 0, s>>>(d);
  }
  if (mode == MODE_CANON) k_after_canon<<<1, 1, 0, s>>>(d);
}

}  // namespace cgdem
