// k_fluid.cu -- two-way coupling by Darcy flow: the fluid of Eq. 6 (model A)
// in the slow-flow limit, where the fluid's momentum balance reduces to
// Darcy's law for the superficial velocity, U = -(K(n) / mu_f) grad p, and
// continuity to div U = 0.  After every porosity update the dynamic pressure
// of the Darcy samples solves div(K grad p) = 0 on the fluid grid (7-point
// finite volumes, harmonic-mean face conductances, the Kozeny-Carman
// permeability of the cell's porosity), the injection pressure held in the
// cells outside the cylinder wall and zero at the outlet, by conjugate
// gradients with the diagonal as preconditioner, in FP64, from the last
// solve's pressure.  Every sum is a fixed-order reduction (per-block partial
// sums, then one block), so the solve is deterministic.
//
// Launch sequence of one solve: k_fl_setup, then the whole iteration in one
// cooperative launch (k_fl_solve: all blocks resident, a bounded grid barrier
// between phases), then k_fl_finish.  Where no cooperative launch can be
// captured, the iteration runs as separate kernels: k_fl_init, k_fl_start,
// then {k_fl_spmv, k_fl_alpha, k_fl_update, k_fl_beta, k_fl_dir} as the body
// of a CUDA-graph WHILE node whose condition k_fl_start and k_fl_beta set (or
// a fixed number of them that return at once once done).  Nothing runs unless
// a porosity update is pending.
#include "cgdem_internal.cuh"

namespace cgdem {

constexpr int FL_B = 256;

__device__ __forceinline__ bool fl_unknown(signed char t) { return t == 0 || t == 3; }

// Cell c's position in its sample's grid; false when the cell is not solved.
struct CellIdx {
  int ijk[3], dim[3], stride[3];
};
__device__ __forceinline__ CellIdx cell_idx(const SampleDev& S, int c) {
  CellIdx ci;
  const int l = c - S.fcell_off;
  ci.dim[0] = S.nf[0];
  ci.dim[1] = S.nf[1];
  ci.dim[2] = S.nf[2];
  ci.ijk[0] = l % S.nf[0];
  ci.ijk[1] = (l / S.nf[0]) % S.nf[1];
  ci.ijk[2] = l / (S.nf[0] * S.nf[1]);
  ci.stride[0] = 1;
  ci.stride[1] = S.nf[0];
  ci.stride[2] = S.nf[0] * S.nf[1];
  return ci;
}

__device__ __forceinline__ double face_area(const SampleDev& S, int k) {
  return S.hf[(k + 1) % 3] * S.hf[(k + 2) % 3];
}
__device__ __forceinline__ double face_cond(const SampleDev& S, int k, double Ka, double Kb) {
  return face_area(S, k) / (S.mu_f * S.hf[k]) * (2.0 * Ka * Kb / (Ka + Kb));
}
__device__ __forceinline__ double outlet_cond(const SampleDev& S, double K) {
  return S.hf[0] * S.hf[1] / (S.mu_f * 0.5 * S.hf[2]) * K;
}

// (A x)_c of an unknown cell; with b, also the right-hand side of the fixed
// pressures around it; with M, the diagonal.
__device__ double apply_A(const Dev& d, const SampleDev& S, int c, const double* x, double* b, double* M) {
  const CellIdx ci = cell_idx(S, c);
  const double Kc = d.fl_K[c];
  double acc = 0.0, rhs = 0.0, dg = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int sg = -1; sg <= 1; sg += 2) {
      const int q = ci.ijk[k] + sg;
      if (q < 0 || q >= ci.dim[k]) continue;
      const int nb = c + sg * ci.stride[k];
      const signed char tn = d.fl_type[nb];
      if (tn == 2) continue;
      const double T = face_cond(S, k, Kc, d.fl_K[nb]);
      dg += T;
      if (fl_unknown(tn)) {
        acc += T * (x[c] - x[nb]);
      } else {
        acc += T * x[c];
        rhs += T * d.fl_p[nb];
      }
    }
  if (d.fl_type[c] == 3) {  // drains to the outlet, p = 0
    const double T = outlet_cond(S, Kc);
    acc += T * x[c];
    dg += T;
  }
  if (b) *b = rhs;
  if (M) *M = dg;
  return acc;
}

// Fixed-order block sum of v (one value per thread) into part[blockIdx.x].
__device__ __forceinline__ void block_partial(double v, double* part) {
  __shared__ double sh[FL_B];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = FL_B / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
  __syncthreads();
}

// Fixed-order sum of n partials by one block; every thread gets it.
__device__ __forceinline__ double block_total(const double* part, int n) {
  __shared__ double sh[FL_B];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += FL_B) v += part[i];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = FL_B / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double t = sh[0];
  __syncthreads();
  return t;
}

// Permeability, the cells' roles, the fixed pressures.
__global__ void __launch_bounds__(FL_B) k_fl_setup(Dev d) {
  if (!d.ctl->fl_pending) return;
  const int c = blockIdx.x * FL_B + threadIdx.x;
  if (c >= d.Cf_total) return;
  const SampleDev& S = d.sp[d.fl_sample[c]];
  if (S.fluid_mode != 1 || S.kind != CGDEM_CYLINDER) {
    d.fl_type[c] = 2;
    return;
  }
  const CellIdx ci = cell_idx(S, c);
  const double xc = S.f_lo[0] + (ci.ijk[0] + 0.5) * S.hf[0];
  const double yc = S.f_lo[1] + (ci.ijk[1] + 0.5) * S.hf[1];
  const double rc = sqrt(xc * xc + yc * yc);
  double n = 1.0 - (double)d.vf[d.ctl->vf_cur][c] * 9.094947017729282379150390625e-13;  // 2^-40
  if (!(n >= S.n_min)) n = S.n_min;
  if (n > 1.0) n = 1.0;
  if (n > DARCY_N_CAP) n = DARCY_N_CAP;
  d.fl_K[c] = S.perm_d2 * n * n * n / ((1.0 - n) * (1.0 - n));
  signed char t = 0;
  if (rc >= S.Rc) {
    t = 1;
    d.fl_p[c] = S.p_inlet;
  } else if (ci.ijk[2] == 0 && rc < S.r_out) {
    t = 3;
  }
  d.fl_type[c] = t;
}

// r = b - A p, z = r / M, d = z; partial sums of r.z, b.b, r.r
__global__ void __launch_bounds__(FL_B) k_fl_init(Dev d) {
  if (!d.ctl->fl_pending) return;
  const int c = blockIdx.x * FL_B + threadIdx.x;
  double rz = 0.0, bb = 0.0, rr = 0.0;
  if (c < d.Cf_total && fl_unknown(d.fl_type[c])) {
    const SampleDev& S = d.sp[d.fl_sample[c]];
    double b, M;
    const double Ap = apply_A(d, S, c, d.fl_p, &b, &M);
    const double r = b - Ap;
    d.fl_M[c] = M;
    d.fl_b[c] = b;
    d.fl_r[c] = r;
    const double z = r / M;
    d.fl_z[c] = z;
    d.fl_d[c] = z;
    rz = r * z;
    bb = b * b;
    rr = r * r;
  }
  block_partial(rz, d.fl_part);
  block_partial(bb, d.fl_part + d.fl_blocks);
  block_partial(rr, d.fl_part + 2 * d.fl_blocks);
}

// Starts a pending solve: the scalars, and the loop's condition.
__global__ void __launch_bounds__(FL_B) k_fl_start(Dev d, cudaGraphConditionalHandle h) {
  Ctl* ctl = d.ctl;
  const int pending = ctl->fl_pending;
  __syncthreads();
  if (!pending) {
    if (threadIdx.x == 0) {
      ctl->fl_done = 1;
      ctl->fl_it = -1;  // no solve: k_fl_finish leaves the field as it is
      if (h) cudaGraphSetConditional(h, 0u);
    }
    return;
  }
  const double rz = block_total(d.fl_part, d.fl_blocks);
  const double bb = block_total(d.fl_part + d.fl_blocks, d.fl_blocks);
  const double rr = block_total(d.fl_part + 2 * d.fl_blocks, d.fl_blocks);
  if (threadIdx.x == 0) {
    ctl->fl_pending = 0;
    ctl->fl_rz = rz;
    ctl->fl_bb = bb;
    ctl->fl_it = 0;
    const int done = rr <= d.fl_tol * d.fl_tol * bb ? 1 : 0;
    ctl->fl_done = done;
    ctl->fl_iters = 0;
    if (h) cudaGraphSetConditional(h, done ? 0u : 1u);
  }
}

// q = A d; partial sums of d.q
__global__ void __launch_bounds__(FL_B) k_fl_spmv(Dev d) {
  if (d.ctl->fl_done) return;
  const int c = blockIdx.x * FL_B + threadIdx.x;
  double dq = 0.0;
  if (c < d.Cf_total && fl_unknown(d.fl_type[c])) {
    const SampleDev& S = d.sp[d.fl_sample[c]];
    const double q = apply_A(d, S, c, d.fl_d, nullptr, nullptr);
    d.fl_q[c] = q;
    dq = d.fl_d[c] * q;
  }
  block_partial(dq, d.fl_part);
}

__global__ void __launch_bounds__(FL_B) k_fl_alpha(Dev d) {
  if (d.ctl->fl_done) return;
  const double dq = block_total(d.fl_part, d.fl_blocks);
  if (threadIdx.x == 0) d.ctl->fl_alpha = d.ctl->fl_rz / dq;
}

// p += alpha d, r -= alpha q, z = r / M; partial sums of r.z and r.r
__global__ void __launch_bounds__(FL_B) k_fl_update(Dev d) {
  if (d.ctl->fl_done) return;
  const double alpha = d.ctl->fl_alpha;
  const int c = blockIdx.x * FL_B + threadIdx.x;
  double rz = 0.0, rr = 0.0;
  if (c < d.Cf_total && fl_unknown(d.fl_type[c])) {
    d.fl_p[c] += alpha * d.fl_d[c];
    const double r = d.fl_r[c] - alpha * d.fl_q[c];
    d.fl_r[c] = r;
    const double z = r / d.fl_M[c];
    d.fl_z[c] = z;
    rz = r * z;
    rr = r * r;
  }
  block_partial(rz, d.fl_part);
  block_partial(rr, d.fl_part + 2 * d.fl_blocks);
}

// Convergence test and the next direction's coefficient; the loop's condition.
__global__ void __launch_bounds__(FL_B) k_fl_beta(Dev d, cudaGraphConditionalHandle h) {
  Ctl* ctl = d.ctl;
  if (ctl->fl_done) {
    if (threadIdx.x == 0 && h) cudaGraphSetConditional(h, 0u);
    return;
  }
  const double rz1 = block_total(d.fl_part, d.fl_blocks);
  const double rr = block_total(d.fl_part + 2 * d.fl_blocks, d.fl_blocks);
  if (threadIdx.x == 0) {
    const int it = ctl->fl_it + 1;
    ctl->fl_it = it;
    unsigned go = 1u;
    if (rr <= d.fl_tol * d.fl_tol * ctl->fl_bb) {
      ctl->fl_done = 1;
      ctl->fl_iters = it;
      go = 0u;
    } else if (it >= d.fl_iters_max) {
      ctl->fl_done = 1;
      ctl->fl_iters = -1;  // stopped short of the tolerance
      go = 0u;
    } else {
      ctl->fl_beta = rz1 / ctl->fl_rz;
      ctl->fl_rz = rz1;
    }
    if (h) cudaGraphSetConditional(h, go);
  }
}

// d = z + beta d
__global__ void __launch_bounds__(FL_B) k_fl_dir(Dev d) {
  if (d.ctl->fl_done) return;
  const double beta = d.ctl->fl_beta;
  const int c = blockIdx.x * FL_B + threadIdx.x;
  if (c < d.Cf_total && fl_unknown(d.fl_type[c])) d.fl_d[c] = d.fl_z[c] + beta * d.fl_d[c];
}

// Superficial velocity (per axis the mean of the cell's two face velocities)
// and the gradient that drives it, -mu_f U / K, of the solved cells.
__global__ void __launch_bounds__(FL_B) k_fl_finish(Dev d) {
  if (d.ctl->fl_it < 0) return;
  const int c = blockIdx.x * FL_B + threadIdx.x;
  if (c >= d.Cf_total) return;
  const signed char t = d.fl_type[c];
  if (t == 2) return;  // a sample without Darcy flow keeps its field
  double U[3] = {0.0, 0.0, 0.0}, G[3] = {0.0, 0.0, 0.0};
  if (fl_unknown(t)) {
    const SampleDev& S = d.sp[d.fl_sample[c]];
    const CellIdx ci = cell_idx(S, c);
    const double Kc = d.fl_K[c], pc = d.fl_p[c];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double u = 0.0;
#pragma unroll
      for (int sg = -1; sg <= 1; sg += 2) {
        const int q = ci.ijk[k] + sg;
        if (q < 0 || q >= ci.dim[k]) continue;
        const int nb = c + sg * ci.stride[k];
        if (d.fl_type[nb] == 2) continue;
        u += sg * face_cond(S, k, Kc, d.fl_K[nb]) * (pc - d.fl_p[nb]) / face_area(S, k);
      }
      if (k == 2 && t == 3) u += -outlet_cond(S, Kc) * pc / face_area(S, 2);
      U[k] = 0.5 * u;
      G[k] = -S.mu_f * U[k] / Kc;
    }
  }
  d.Us[c] = make_double4(U[0], U[1], U[2], 0.0);
  d.Usf[c] = make_float4((float)U[0], (float)U[1], (float)U[2], 0.f);
  d.gradp[c] = make_double4(G[0], G[1], G[2], 0.0);
  d.gradpf[c] = make_float4((float)G[0], (float)G[1], (float)G[2], 0.f);
}

// ---- the whole solve in one cooperative launch ----------------------------
//
// The same iteration in one launch whose blocks are all resident: each block
// takes a fixed set of cells (grid stride), writes its partial sums, and a
// grid barrier separates the phases; after a barrier every block forms the
// same totals from the partials in the same order, so all blocks take the
// same decisions and the result does not depend on timing.  Two barriers per
// iteration: the new direction d = z + beta d_old is formed on the fly where
// A d needs it (neighbours included), into a second buffer, so that nobody
// overwrites a direction another block still reads.
constexpr int FL_WAIT_LIMIT = 1 << 21;  // polls of a barrier before the solve gives up

// Grid barrier: one arrival per block; the last to arrive opens the next
// generation.  false when the wait gave up (the solve is then abandoned and
// the step latches a timeout).
__device__ __forceinline__ bool fl_grid_sync(Ctl* ctl, unsigned& gen) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    const unsigned a = atomicAdd(&ctl->fl_bar_count, 1u);
    if (a == gridDim.x - 1u) {
      atomicExch(&ctl->fl_bar_count, 0u);
      __threadfence();
      atomicExch(&ctl->fl_bar_gen, gen + 1u);
    } else {
      int polls = 0;
      while (*((volatile unsigned*)&ctl->fl_bar_gen) == gen) {
        if (++polls > FL_WAIT_LIMIT || *((volatile int*)&ctl->fl_abort)) {
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (!ok) {
      atomicExch(&ctl->fl_abort, 1);
      latch(ctl, ST_TIMEOUT);
    }
    ok_s = ok;
  }
  __syncthreads();
  gen += 1u;
  return ok_s != 0;
}

// Direction entry i of this iteration, z_i + beta d_old,i: the owner and its
// neighbours evaluate the same expression on the same values.
__device__ __forceinline__ double fl_dir(const double* z, const double* dold, double beta, int i) {
  return __fma_rn(beta, dold[i], z[i]);
}

// Conductances of cell c's upper faces (x, y, z) and of its outlet face,
// from the permeabilities of k_fl_setup; 0 where the neighbour is not part
// of the system.  face_cond is symmetric in its two permeabilities, so each
// face gets the value either side would compute.
__device__ double4 face_conds(const Dev& d, const SampleDev& S, int c) {
  const CellIdx ci = cell_idx(S, c);
  const double Kc = d.fl_K[c];
  double T[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (ci.ijk[k] + 1 >= ci.dim[k]) continue;
    const int nb = c + ci.stride[k];
    if (d.fl_type[nb] == 2) continue;
    T[k] = face_cond(S, k, Kc, d.fl_K[nb]);
  }
  const double To = d.fl_type[c] == 3 ? outlet_cond(S, Kc) : 0.0;
  return make_double4(T[0], T[1], T[2], To);
}

// (A x)_c of an unknown cell from the stored conductances, where x_i =
// z_i + beta d_old,i (dold == nullptr: x = z); with b and M, also the
// right-hand side of the fixed pressures around it and the diagonal.  The
// terms are added in the order apply_A adds them.
__device__ double apply_A_stored(const Dev& d, const SampleDev& S, int c, const double* z, const double* dold,
                                 double beta, double* xc_out, double* b, double* M) {
  const CellIdx ci = cell_idx(S, c);
  const double4 Tc = d.fl_T[c];
  const double Tup[3] = {Tc.x, Tc.y, Tc.z};
  const double xc = dold ? fl_dir(z, dold, beta, c) : z[c];
  double acc = 0.0, rhs = 0.0, dg = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int sg = -1; sg <= 1; sg += 2) {
      const int q = ci.ijk[k] + sg;
      if (q < 0 || q >= ci.dim[k]) continue;
      const int nb = c + sg * ci.stride[k];
      const signed char tn = d.fl_type[nb];
      if (tn == 2) continue;
      double T;
      if (sg < 0) {
        const double4 Tn = d.fl_T[nb];
        T = k == 0 ? Tn.x : (k == 1 ? Tn.y : Tn.z);
      } else {
        T = Tup[k];
      }
      dg += T;
      if (fl_unknown(tn)) {
        acc += T * (xc - (dold ? fl_dir(z, dold, beta, nb) : z[nb]));
      } else {
        acc += T * xc;
        rhs += T * d.fl_p[nb];
      }
    }
  if (d.fl_type[c] == 3) {
    acc += Tc.w * xc;
    dg += Tc.w;
  }
  if (xc_out) *xc_out = xc;
  if (b) *b = rhs;
  if (M) *M = dg;
  return acc;
}

// Fixed-order block sums of up to three values per thread into part[k * G + blockIdx.x].
__device__ __forceinline__ void block_partials(double a, double b, double c, int nv, double* part, int G) {
  __shared__ double sh[3][FL_B];
  sh[0][threadIdx.x] = a;
  sh[1][threadIdx.x] = b;
  sh[2][threadIdx.x] = c;
  __syncthreads();
  for (int o = FL_B / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int k = 0; k < nv; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + o];
    __syncthreads();
  }
  if ((int)threadIdx.x < nv) part[threadIdx.x * G + blockIdx.x] = sh[threadIdx.x][0];
  __syncthreads();
}

__global__ void __launch_bounds__(FL_B) k_fl_solve(Dev d) {
  Ctl* ctl = d.ctl;
  // every block reads the flag before the first barrier; block 0 clears it after
  const int pending = *((volatile int*)&ctl->fl_pending);
  if (!pending) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      ctl->fl_done = 1;
      ctl->fl_it = -1;  // no solve: k_fl_finish leaves the field as it is
    }
    return;
  }
  unsigned gen = atomicAdd(&ctl->fl_bar_gen, 0u);
  const int G = (int)gridDim.x;
  const int c0 = blockIdx.x * FL_B + threadIdx.x, cs = G * FL_B;
  double* part = d.fl_part;  // slots of G partials: r.z, b.b (then r.r), r.r, d.q
  const double tol2 = d.fl_tol * d.fl_tol;
  // the face conductances of this solve's permeabilities, once
  for (int c = c0; c < d.Cf_total; c += cs) {
    if (d.fl_type[c] == 2) continue;
    d.fl_T[c] = face_conds(d, d.sp[d.fl_sample[c]], c);
  }
  if (!fl_grid_sync(ctl, gen)) return;
  // r = b - A p, z = r / M; the first direction is z (d_old = 0, beta = 0)
  double rz = 0.0, bb = 0.0, rr = 0.0;
  for (int c = c0; c < d.Cf_total; c += cs) {
    if (!fl_unknown(d.fl_type[c])) continue;
    const SampleDev& S = d.sp[d.fl_sample[c]];
    double b, M;
    const double Ap = apply_A_stored(d, S, c, d.fl_p, nullptr, 0.0, nullptr, &b, &M);
    const double rc = b - Ap;
    const double z = rc / M;
    d.fl_M[c] = M;
    d.fl_r[c] = rc;
    d.fl_z[c] = z;
    d.fl_d[c] = 0.0;
    rz += rc * z;
    bb += b * b;
    rr += rc * rc;
  }
  block_partials(rz, bb, rr, 3, part, G);
  if (!fl_grid_sync(ctl, gen)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->fl_pending = 0;
  double rzt = block_total(part, G);
  const double bbt = block_total(part + G, G);
  double rrt = block_total(part + 2 * G, G);
  int it = 0;
  long long iters = 0;
  bool done = rrt <= tol2 * bbt;
  double beta = 0.0;
  double* dold = d.fl_d;
  double* dnew = d.fl_d2;
  while (!done) {
    // q = A d with d = z + beta d_old; d.q
    double dq = 0.0;
    for (int c = c0; c < d.Cf_total; c += cs) {
      if (!fl_unknown(d.fl_type[c])) continue;
      const SampleDev& S = d.sp[d.fl_sample[c]];
      double dc;
      const double q = apply_A_stored(d, S, c, d.fl_z, dold, beta, &dc, nullptr, nullptr);
      dnew[c] = dc;
      d.fl_q[c] = q;
      dq += dc * q;
    }
    block_partials(dq, 0.0, 0.0, 1, part + 3 * G, G);
    if (!fl_grid_sync(ctl, gen)) return;
    const double alpha = rzt / block_total(part + 3 * G, G);
    // p += alpha d, r -= alpha q, z = r / M; r.z and r.r
    double rz1 = 0.0, rr1 = 0.0;
    for (int c = c0; c < d.Cf_total; c += cs) {
      if (!fl_unknown(d.fl_type[c])) continue;
      d.fl_p[c] += alpha * dnew[c];
      const double r = d.fl_r[c] - alpha * d.fl_q[c];
      d.fl_r[c] = r;
      const double z = r / d.fl_M[c];
      d.fl_z[c] = z;
      rz1 += r * z;
      rr1 += r * r;
    }
    block_partials(rz1, rr1, 0.0, 2, part, G);  // slot 1 is free once b.b is summed
    if (!fl_grid_sync(ctl, gen)) return;
    const double rzn = block_total(part, G);
    rrt = block_total(part + G, G);
    ++it;
    if (rrt <= tol2 * bbt) {
      done = true;
      iters = it;
    } else if (it >= d.fl_iters_max) {
      done = true;
      iters = -1;  // stopped short of the tolerance
    } else {
      beta = rzn / rzt;
      rzt = rzn;
      double* t = dold;
      dold = dnew;
      dnew = t;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->fl_done = 1;
    ctl->fl_it = it;
    ctl->fl_iters = iters;
  }
}

__global__ void k_fl_mark(Dev d) { d.ctl->fl_pending = 1; }

// the drag-reaction buffer of a force evaluation at the current step
__global__ void k_react_clear(Dev d) {
  unsigned long long* z = d.react[d.ctl->step & 1];
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < 3 * d.Cf_total; c += gridDim.x * blockDim.x)
    z[c] = 0ull;
}

static inline int fl_grid(const Dev& d) { return (d.Cf_total + FL_B - 1) / FL_B; }

void launch_fluid_mark(const Dev& d, cudaStream_t s) { k_fl_mark<<<1, 1, 0, s>>>(d); }

void launch_react_clear(const Dev& d, cudaStream_t s) { k_react_clear<<<fl_grid(d), FL_B, 0, s>>>(d); }

void launch_fluid_head(const Dev& d, cudaGraphConditionalHandle h, cudaStream_t s) {
  const int G = fl_grid(d);
  k_fl_setup<<<G, FL_B, 0, s>>>(d);
  k_fl_init<<<G, FL_B, 0, s>>>(d);
  k_fl_start<<<1, FL_B, 0, s>>>(d, h);
}

void launch_fluid_iteration(const Dev& d, cudaGraphConditionalHandle h, cudaStream_t s) {
  const int G = fl_grid(d);
  k_fl_spmv<<<G, FL_B, 0, s>>>(d);
  k_fl_alpha<<<1, FL_B, 0, s>>>(d);
  k_fl_update<<<G, FL_B, 0, s>>>(d);
  k_fl_beta<<<1, FL_B, 0, s>>>(d, h);
  k_fl_dir<<<G, FL_B, 0, s>>>(d);
}

void launch_fluid_tail(const Dev& d, cudaStream_t s) { k_fl_finish<<<fl_grid(d), FL_B, 0, s>>>(d); }

int fluid_blocks(int Cf_total) { return (Cf_total + FL_B - 1) / FL_B; }

// Blocks of the one-launch solve: two per SM, no more than the cells need and
// no more than can be resident at once; 0 when no cooperative launch is
// possible (the WHILE-node form is used then).
int fluid_coop_blocks(int Cf_total) {
  int dev = 0, sms = 0, coop = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fl_solve, FL_B, 0) != cudaSuccess) return 0;
  if (per_sm < 1) return 0;
  int G = 2 * sms;
  if (G > per_sm * sms) G = per_sm * sms;
  const int need = fluid_blocks(Cf_total);
  if (G > need) G = need;
  return G > 0 ? G : 0;
}

// One solve as three launches: setup, the cooperative solve, the velocity.
cudaError_t launch_fluid_solve_coop(const Dev& d, cudaStream_t s) {
  k_fl_setup<<<fl_grid(d), FL_B, 0, s>>>(d);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)d.fl_coop_blocks);
  cfg.blockDim = dim3(FL_B);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_fl_solve, d);
  if (e != cudaSuccess) return e;
  k_fl_finish<<<fl_grid(d), FL_B, 0, s>>>(d);
  return cudaGetLastError();
}

}  // namespace cgdem
