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
// Launch sequence of one solve: k_fl_setup, k_fl_init, k_fl_start, then the
// iterations {k_fl_spmv, k_fl_alpha, k_fl_update, k_fl_beta, k_fl_dir} --
// the body of a CUDA-graph WHILE node whose condition k_fl_start and
// k_fl_beta set (or a fixed number of them that return at once once done),
// then k_fl_finish.  Nothing runs unless a porosity update is pending.
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

}  // namespace cgdem
