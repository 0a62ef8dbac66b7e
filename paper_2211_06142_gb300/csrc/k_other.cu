// k_other.cu -- candidate-list rebuild (cell binning, deterministic counting
// sort, permutation, neighbour-cell scan with history carry), porosity
// scatter, velocity-Verlet halves, initial state and readback kernels.
#include "cgdem_internal.cuh"

namespace cgdem {

// ---------------------------------------------------------------------------
// rebuild: bin -> scan -> scatter -> rank -> permute -> search -> finish
// Every kernel returns at once unless ctl->rebuild is set, so the sequence
// can sit in a CUDA graph and only costs launches on steps without rebuild.
// ---------------------------------------------------------------------------

__global__ void k_rb_bin(Dev d) {
  if (!d.ctl->rebuild) return;
  const int cur = d.ctl->cur, pc = d.ctl->pcur;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= d.N) return;
  double4 P = d.pos[cur][p];
  uint32_t c;
  if (P.w > 0.0) {
    int cxyz[3];
    c = (uint32_t)search_cell_of(d.sp[d.sample[pc][p]], P.x, P.y, P.z, cxyz);
  } else {
    c = (uint32_t)d.C_total;  // particles that left: one bin after all cells
  }
  d.pcell[p] = c;
  d.pslot[p] = atomicAdd(&d.cell_count[c], 1u);
}

// Exclusive scan of cell_count[0..C] into cell_start[0..C+1] in three passes
// (tile sums, scan of the tile sums, tile scans), clearing the counts.
constexpr int SCAN_T = 256, SCAN_V = 8, SCAN_TILE = SCAN_T * SCAN_V;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* warp_sums,
                                                         uint32_t* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_sums[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = lane < nw ? warp_sums[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) warp_sums[lane] = w;
  }
  __syncthreads();
  const uint32_t before = wid > 0 ? warp_sums[wid - 1] : 0u;
  *total = warp_sums[nw - 1];
  __syncthreads();
  return before + incl - x;
}

__global__ void __launch_bounds__(SCAN_T) k_rb_scan_tiles(Dev d, uint32_t* tile_sums) {
  if (!d.ctl->rebuild) return;
  __shared__ uint32_t ws[32];
  const int n = d.C_total + 1;
  const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_V;
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < SCAN_V; ++j) s += base + j < n ? d.cell_count[base + j] : 0u;
  uint32_t tot;
  block_exclusive_scan(s, ws, &tot);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_rb_scan_sums(Dev d, uint32_t* tile_sums, int ntiles) {
  if (!d.ctl->rebuild) return;
  __shared__ uint32_t ws[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < ntiles; b0 += 1024) {
    const int i = b0 + threadIdx.x;
    const uint32_t v = i < ntiles ? tile_sums[i] : 0u;
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan(v, ws, &tot);
    if (i < ntiles) tile_sums[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) d.cell_start[d.C_total + 1] = carry;
}

__global__ void __launch_bounds__(SCAN_T) k_rb_scan_apply(Dev d, const uint32_t* tile_sums) {
  if (!d.ctl->rebuild) return;
  __shared__ uint32_t ws[32];
  const int n = d.C_total + 1;
  const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_V;
  uint32_t v[SCAN_V];
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < SCAN_V; ++j) {
    v[j] = base + j < n ? d.cell_count[base + j] : 0u;
    s += v[j];
  }
  uint32_t tot;
  uint32_t ex = block_exclusive_scan(s, ws, &tot) + tile_sums[blockIdx.x];
#pragma unroll
  for (int j = 0; j < SCAN_V; ++j) {
    if (base + j < n) {
      d.cell_start[base + j] = ex;
      d.cell_count[base + j] = 0u;
    }
    ex += v[j];
  }
}

__global__ void k_rb_scatter(Dev d) {
  if (!d.ctl->rebuild) return;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= d.N) return;
  d.perm_tmp[d.cell_start[d.pcell[p]] + d.pslot[p]] = (uint32_t)p;
}

// Deterministic order inside each cell: rank by particle id.
__global__ void k_rb_rank(Dev d) {
  if (!d.ctl->rebuild) return;
  const int pc = d.ctl->pcur;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= d.N) return;
  const uint32_t i = d.perm_tmp[q];
  const uint32_t c = d.pcell[i];
  const uint32_t s0 = d.cell_start[c], s1 = d.cell_start[c + 1];
  if (c == (uint32_t)d.C_total) {  // particles that left: order is irrelevant
    d.perm[q] = i;
    return;
  }
  const int myid = d.id[pc][i];
  uint32_t rank = 0;
  for (uint32_t j = s0; j < s1; ++j) rank += d.id[pc][d.perm_tmp[j]] < myid ? 1u : 0u;
  d.perm[s0 + rank] = i;
}

// Gather every per-particle array into the other buffer in the new order.
__global__ void k_rb_permute(Dev d) {
  if (!d.ctl->rebuild) return;
  const int cur = d.ctl->cur, nxt = cur ^ 1;
  const int pc = d.ctl->pcur, pn = pc ^ 1;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= d.N) return;
  const uint32_t o = d.perm[p];
  d.inv_perm[o] = (uint32_t)p;
  d.cand_n[p] = 0u;
  if (p == 0) *d.big_n = 0u;
  double4 P = d.pos[cur][o];
  d.pos[nxt][p] = P;
  d.vel[nxt][p] = d.vel[cur][o];
  d.omg[nxt][p] = d.omg[cur][o];
  const int s = d.sample[pc][o];
  const SampleDev& S = d.sp[s];
  int4 q;
  q.x = to_q(P.x, S.inv_dq);
  q.y = to_q(P.y, S.inv_dq);
  q.z = to_q(P.z, S.inv_dq);
  q.w = P.w > 0.0 ? d.posq[cur][o].w : 0;
  d.posq[nxt][p] = q;
  d.velf[nxt][p] = d.velf[cur][o];
  d.omgf[nxt][p] = d.omgf[cur][o];
  d.id[pn][p] = d.id[pc][o];
  d.sample[pn][p] = s;
  d.fcell[pn][p] = d.fcell[pc][o];
  d.vq[pn][p] = d.vq[pc][o];
  if (d.clc[0]) d.clc[nxt][p] = d.clc[cur][o];
  if (d.mixed && d.wallhf[0]) {
    for (int w = 0; w < CGDEM_WALLS; ++w)
      d.wallhf[pn][(size_t)w * d.Npad + p] = d.wallhf[pc][(size_t)w * d.Npad + o];
  } else if (!d.mixed && d.wallh[0]) {
    for (int w = 0; w < CGDEM_WALLS; ++w)
      d.wallh[pn][(size_t)w * d.Npad + p] = d.wallh[pc][(size_t)w * d.Npad + o];
  }
}

// Permute the single-buffered force and torque through staging memory.
__global__ void k_rb_ft_gather(Dev d) {
  if (!d.ctl->rebuild) return;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= d.N) return;
  const uint32_t o = d.perm[p];
  double4* st = reinterpret_cast<double4*>(d.staging);
  st[p] = d.F[o];
  st[d.Npad + p] = d.T[o];
}
__global__ void k_rb_ft_store(Dev d) {
  if (!d.ctl->rebuild) return;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= d.N) return;
  const double4* st = reinterpret_cast<const double4*>(d.staging);
  const uint32_t c = d.mixed ? d.sched[p] : (uint32_t)p;  // mixed: schedule order
  d.F[p] = st[c];
  d.T[p] = st[d.Npad + c];
}

constexpr int BIG_STENCIL = 27;  // stencils of more than 3^3 cells are walked by a warp

// Candidate pairs: d^2 < (Ri + Rj + skin)^2 in fixed point (exact integer
// test).  Each pair is found once, from its larger sphere (ties: higher
// index), whose stencil (2 R + skin) covers the pair whatever the partner's
// size; the cell edge can then follow the typical rather than the largest
// sphere.  The pair goes into both spheres' lists (atomic slots); the lists
// are sorted by partner afterwards, so the result does not depend on the
// order of the atomics.
__global__ void k_rb_pairs(Dev d) {
  if (!d.ctl->rebuild) return;
  const int nxt = d.ctl->cur ^ 1;
  const int pn = d.ctl->pcur ^ 1;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= d.N) return;
  const int4 pq = d.posq[nxt][p];
  if (pq.w <= 0) return;
  const int Npad = d.Npad, cap = d.cap;
  const int s = d.sample[pn][p];
  const SampleDev& S = d.sp[s];
  const uint32_t o = d.perm[p];
  const int lc = (int)d.pcell[o] - S.cell_off;
  const int cc[3] = {lc % S.nc[0], (lc / S.nc[0]) % S.nc[1], lc / (S.nc[0] * S.nc[1])};
  const bool per = S.kind == CGDEM_PERIODIC_BOX;
  const float reach = 2.0f * (float)pq.w * S.dq_f + S.skin_f;
  int lo[3], hi[3];
  bool all[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int r = (int)ceilf(reach * S.c_inv_h_f[k] * 1.000001f);
    all[k] = per && 2 * r + 1 >= S.nc[k];
    lo[k] = all[k] ? 0 : cc[k] - r;
    hi[k] = all[k] ? S.nc[k] - 1 : cc[k] + r;
    if (!per) {
      lo[k] = max(lo[k], 0);
      hi[k] = min(hi[k], S.nc[k] - 1);
    }
  }
  const unsigned long long skin_q = (unsigned)S.skin_q;
  // a large sphere's stencil is walked by a whole warp in k_rb_pairs_big:
  // its cells are serial dependent loads, and one thread would set the
  // kernel's time
  if ((hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1) > BIG_STENCIL) {
    d.big_list[atomicAdd(d.big_n, 1u)] = (uint32_t)p;
    return;
  }
  // The cells of a stencil row (fixed y, z) are consecutive in the cell
  // order, so their spheres are one index range (two where a periodic row
  // wraps): one pair of cell_start loads per row instead of per cell.
  int xs[2], xe[2], nseg = 1;
  xs[0] = lo[0];
  xe[0] = hi[0];
  if (per && !all[0]) {
    if (lo[0] < 0) {
      xs[0] = lo[0] + S.nc[0], xe[0] = S.nc[0] - 1, xs[1] = 0, xe[1] = hi[0], nseg = 2;
    } else if (hi[0] >= S.nc[0]) {
      xs[0] = lo[0], xe[0] = S.nc[0] - 1, xs[1] = 0, xe[1] = hi[0] - S.nc[0], nseg = 2;
    }
  }
  for (int az = lo[2]; az <= hi[2]; ++az) {
    const int z = per && !all[2] ? (az + S.nc[2]) % S.nc[2] : az;
    for (int ay = lo[1]; ay <= hi[1]; ++ay) {
      const int y = per && !all[1] ? (ay + S.nc[1]) % S.nc[1] : ay;
      const int row = S.cell_off + (z * S.nc[1] + y) * S.nc[0];
      for (int sgm = 0; sgm < nseg; ++sgm) {
        const uint32_t j0 = d.cell_start[row + xs[sgm]], j1 = d.cell_start[row + xe[sgm] + 1];
#pragma unroll 4
        for (uint32_t q = j0; q < j1; ++q) {
          const int4 qq = d.posq[nxt][q];
          if (qq.w <= 0) continue;
          if (qq.w > pq.w || (qq.w == pq.w && (int)q <= p)) continue;  // found by the larger one
          const int dx = (int)((uint32_t)qq.x - (uint32_t)pq.x);
          const int dy = (int)((uint32_t)qq.y - (uint32_t)pq.y);
          const int dz = (int)((uint32_t)qq.z - (uint32_t)pq.z);
          const unsigned long long d2 = (unsigned long long)((long long)dx * dx) +
                                        (unsigned long long)((long long)dy * dy) +
                                        (unsigned long long)((long long)dz * dz);
          const unsigned long long Sq = (unsigned long long)(unsigned)pq.w + (unsigned)qq.w + skin_q;
          if (d2 < Sq * Sq) {
            const uint32_t a = atomicAdd(&d.cand_n[p], 1u);
            if (a < (uint32_t)cap) d.cand_tmp[(size_t)a * Npad + p] = q;
            const uint32_t b = atomicAdd(&d.cand_n[q], 1u);
            if (b < (uint32_t)cap) d.cand_tmp[(size_t)b * Npad + q] = (uint32_t)p;
          }
        }
      }
    }
  }
}

// Candidate pairs of the large spheres deferred by k_rb_pairs: one warp per
// sphere, the lanes sharing its stencil cells.
__global__ void k_rb_pairs_big(Dev d) {
  if (!d.ctl->rebuild) return;
  const int nxt = d.ctl->cur ^ 1;
  const int pn = d.ctl->pcur ^ 1;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int nbig = (int)*d.big_n;
  const int Npad = d.Npad, cap = d.cap;
  for (int b = gw; b < nbig; b += nw) {
    const int p = (int)d.big_list[b];
    const int4 pq = d.posq[nxt][p];
    const SampleDev& S = d.sp[d.sample[pn][p]];
    const uint32_t o = d.perm[p];
    const int lc = (int)d.pcell[o] - S.cell_off;
    const int cc[3] = {lc % S.nc[0], (lc / S.nc[0]) % S.nc[1], lc / (S.nc[0] * S.nc[1])};
    const bool per = S.kind == CGDEM_PERIODIC_BOX;
    const float reach = 2.0f * (float)pq.w * S.dq_f + S.skin_f;
    int lo[3], ext[3];
    bool all[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int r = (int)ceilf(reach * S.c_inv_h_f[k] * 1.000001f);
      all[k] = per && 2 * r + 1 >= S.nc[k];
      int l = all[k] ? 0 : cc[k] - r;
      int h = all[k] ? S.nc[k] - 1 : cc[k] + r;
      if (!per) {
        l = max(l, 0);
        h = min(h, S.nc[k] - 1);
      }
      lo[k] = l;
      ext[k] = h - l + 1;
    }
    const unsigned long long skin_q = (unsigned)S.skin_q;
    // lanes take the stencil's rows of cells (fixed y, z), each one index
    // range of the cell-sorted spheres (two where a periodic row wraps)
    int xs[2], xe[2], nseg = 1;
    xs[0] = lo[0];
    xe[0] = lo[0] + ext[0] - 1;
    if (per && !all[0]) {
      if (xs[0] < 0) {
        xs[1] = 0, xe[1] = xe[0], xs[0] += S.nc[0], xe[0] = S.nc[0] - 1, nseg = 2;
      } else if (xe[0] >= S.nc[0]) {
        xs[1] = 0, xe[1] = xe[0] - S.nc[0], xe[0] = S.nc[0] - 1, nseg = 2;
      }
    }
    const int total = ext[1] * ext[2] * nseg;
    for (int t = lane; t < total; t += 32) {
      const int sgm = t % nseg, r = t / nseg;
      const int ay = lo[1] + r % ext[1];
      const int az = lo[2] + r / ext[1];
      const int y = per && !all[1] ? (ay + S.nc[1]) % S.nc[1] : ay;
      const int z = per && !all[2] ? (az + S.nc[2]) % S.nc[2] : az;
      const int row = S.cell_off + (z * S.nc[1] + y) * S.nc[0];
      const uint32_t j0 = d.cell_start[row + xs[sgm]], j1 = d.cell_start[row + xe[sgm] + 1];
#pragma unroll 4
      for (uint32_t q = j0; q < j1; ++q) {
        const int4 qq = d.posq[nxt][q];
        if (qq.w <= 0) continue;
        if (qq.w > pq.w || (qq.w == pq.w && (int)q <= p)) continue;
        const int dx = (int)((uint32_t)qq.x - (uint32_t)pq.x);
        const int dy = (int)((uint32_t)qq.y - (uint32_t)pq.y);
        const int dz = (int)((uint32_t)qq.z - (uint32_t)pq.z);
        const unsigned long long d2 = (unsigned long long)((long long)dx * dx) +
                                      (unsigned long long)((long long)dy * dy) +
                                      (unsigned long long)((long long)dz * dz);
        const unsigned long long Sq = (unsigned long long)(unsigned)pq.w + (unsigned)qq.w + skin_q;
        if (d2 < Sq * Sq) {
          const uint32_t a = atomicAdd(&d.cand_n[p], 1u);
          if (a < (uint32_t)cap) d.cand_tmp[(size_t)a * Npad + p] = q;
          const uint32_t bq = atomicAdd(&d.cand_n[q], 1u);
          if (bq < (uint32_t)cap) d.cand_tmp[(size_t)bq * Npad + q] = (uint32_t)p;
        }
      }
    }
  }
}

// Mixed: the force kernel's schedule.  Per tile of SCHED_TILE consecutive
// spheres (cell order, so a tile is a compact region of the sample), the
// spheres are ordered by decreasing candidate count, spheres of equal count
// in cell order (a stable counting sort: the slots, and so the order of
// every list, are the same on every run), and dealt to consecutive slots;
// slot s is lane s % ppw of the force kernel's warp s / ppw, whose records
// are entry-major: entry k of that lane's sphere at
// (s / ppw) ppw cap + k ppw + s % ppw.
constexpr int SCHED_TILE = 1024;
__global__ void __launch_bounds__(SCHED_TILE) k_rb_sched(Dev d) {
  if (!d.ctl->rebuild) return;
  const int rn = d.ctl->rec_cur ^ 1;
  constexpr int NW = SCHED_TILE / 32, NK = CGDEM_MAX_NEIGHBORS + 1;
  __shared__ uint32_t wpre[NW][NK];  // per warp and count: spheres, then the earlier warps' spheres
  __shared__ uint32_t start[NK];     // per count: spheres, then the first slot
  const int cap = d.cap, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < NW * NK; i += blockDim.x) (&wpre[0][0])[i] = 0u;
  __syncthreads();
  const int t0 = blockIdx.x * SCHED_TILE;
  const int p = t0 + (int)threadIdx.x;
  const bool valid = p < d.N;
  const uint32_t n = valid ? min(d.cand_n[p], (uint32_t)cap) : 0u;
  const uint32_t key = valid ? (uint32_t)cap - n : 0xffffffffu;  // larger lists first
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const uint32_t rank = __popc(peers & ((1u << lane) - 1u));  // earlier lanes with this count
  if (valid && rank == 0) wpre[wid][key] = __popc(peers);
  __syncthreads();
  if ((int)threadIdx.x <= cap) {
    uint32_t run = 0u;
    for (int w = 0; w < NW; ++w) {
      const uint32_t c = wpre[w][threadIdx.x];
      wpre[w][threadIdx.x] = run;
      run += c;
    }
    start[threadIdx.x] = run;
  }
  __syncthreads();
  if (threadIdx.x < 32) {  // exclusive scan of the cap + 1 <= 97 counts: 4 per lane
    uint32_t v[4], sum = 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int b = 4 * lane + j;
      v[j] = b <= cap ? start[b] : 0u;
      sum += v[j];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    uint32_t run = incl - sum;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int b = 4 * lane + j;
      if (b <= cap) start[b] = run;
      run += v[j];
    }
  }
  __syncthreads();
  if (valid) {
    const uint32_t slot = (uint32_t)t0 + start[key] + wpre[wid][key] + rank;
    d.sched[slot] = (uint32_t)p;
    d.perm_tmp[p] = slot;  // cell-order index -> slot (free after k_rb_rank)
  } else if (p < d.Npad) {
    d.sched[p] = 0xffffffffu;  // the slots after the last sphere
  }
  if (p < d.Npad) {
    const uint32_t P = (uint32_t)d.ppw, sl = (uint32_t)p;
    d.roff[rn][sl] = (sl / P) * P * (uint32_t)cap + (sl & (P - 1u));
  }
}

// Mixed: gather every per-particle array from cell order (the buffers the
// first permutation filled) into schedule order (back into the current
// buffers), so that the force kernel's warps read and write their spheres'
// data in consecutive lines.  Slot s holds the sphere of cell-order index
// sched[s].
__global__ void k_rb_permute2(Dev d) {
  if (!d.ctl->rebuild) return;
  const int cur = d.ctl->cur, nxt = cur ^ 1;
  const int pc = d.ctl->pcur, pn = pc ^ 1;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= d.N) return;
  const uint32_t c = d.sched[s];
  d.pos[cur][s] = d.pos[nxt][c];
  d.vel[cur][s] = d.vel[nxt][c];
  d.omg[cur][s] = d.omg[nxt][c];
  d.posq[cur][s] = d.posq[nxt][c];
  d.velf[cur][s] = d.velf[nxt][c];
  d.omgf[cur][s] = d.omgf[nxt][c];
  d.id[pc][s] = d.id[pn][c];
  d.sample[pc][s] = d.sample[pn][c];
  d.fcell[pc][s] = d.fcell[pn][c];
  d.vq[pc][s] = d.vq[pn][c];
  if (d.clc[0]) d.clc[cur][s] = d.clc[nxt][c];
  if (d.wallhf[0])
    for (int w = 0; w < CGDEM_WALLS; ++w)
      d.wallhf[pc][(size_t)w * d.Npad + s] = d.wallhf[pn][(size_t)w * d.Npad + c];
}

// Mixed: every sphere lists all its candidates.  Per slot (the sphere's
// index in schedule order), sort its list by partner (partners in schedule
// order), write it at the slot's records (entry-major per warp) and carry the
// contact history of the old records by particle pair.
__global__ void k_rb_lists_full(Dev d) {
  if (!d.ctl->rebuild) return;
  const int cur = d.ctl->cur;  // the new state, in schedule order (k_rb_permute2)
  const int pc = d.ctl->pcur;
  const int rc = d.ctl->rec_cur, rn = rc ^ 1;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;  // slot; the grid covers Npad exactly
  const int lane = threadIdx.x & 31;
  const int Npad = d.Npad, cap = d.cap;
  if (p - lane >= Npad) return;  // whole warps only (Npad is a multiple of 256)
  const bool valid = p < d.N;
  const uint32_t c = valid ? d.sched[p] : 0u;  // cell-order index of the slot's sphere
  uint32_t count = valid ? d.cand_n[c] : 0u;
  if (count > (uint32_t)cap) latch(d.ctl, ST_CAPACITY);
  unsigned mx = count, sum = count;
#pragma unroll
  for (int k = 16; k >= 1; k >>= 1) {
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, k));
    sum += __shfl_xor_sync(0xffffffffu, sum, k);
  }
  if (lane == 0 && sum) {
    atomicMax(&d.ctl->max_cand_next, (int)mx);
    atomicAdd((unsigned long long*)&d.ctl->cand_total_next, (unsigned long long)sum);
  }
  const uint32_t n = count < (uint32_t)cap ? count : (uint32_t)cap;
  d.cnt[rn][p] = n;
  if (!valid) return;
  const size_t first = d.roff[rn][p];
  const size_t rs = (size_t)d.rstride;
  const int4 pq = d.posq[cur][p];
  d.posq_ref[p] = pq;
  // insertion sort by partner slot (lists are short; sizes vary with the PSD)
  uint32_t lst[CGDEM_MAX_NEIGHBORS];
  for (uint32_t j = 0; j < n; ++j) {
    const uint32_t v = d.perm_tmp[d.cand_tmp[(size_t)j * Npad + c]];
    uint32_t i = j;
    while (i > 0 && lst[i - 1] > v) {
      lst[i] = lst[i - 1];
      --i;
    }
    lst[i] = v;
  }
  uint4* recs = reinterpret_cast<uint4*>(d.rec[rn]);
  for (uint32_t j = 0; j < n; ++j) recs[first + j * rs] = make_uint4(lst[j], 0u, 0u, 0u);
  if (pq.w <= 0) return;
  // carry history: old records of this particle with any state; an old
  // index maps to its cell-order index (inv_perm), then to its slot
  uint32_t carried[(CGDEM_MAX_NEIGHBORS + 31) / 32] = {};  // entries that received a state
  const uint32_t o = d.perm[c];
  const uint32_t nold = d.cnt[rc][o];
  const size_t oldfirst = d.roff[rc][o];
  const uint4* orecs = reinterpret_cast<const uint4*>(d.rec[rc]);
  for (uint32_t k = 0; k < nold; ++k) {
    const uint4 rf = orecs[oldfirst + k * rs];
    const uint32_t pf = rf.x;
    const bool nz = (rf.y | rf.z | rf.w) != 0u;
    if (!(pf & (REC_BOND | REC_ACTIVE)) && !nz) continue;
    const uint32_t qn = d.perm_tmp[d.inv_perm[pf & REC_IDX]];
    // binary search in the sorted list
    int a = 0, b = (int)n - 1, hit = -1;
    while (a <= b) {
      const int m = (a + b) >> 1;
      if (lst[m] == qn) {
        hit = m;
        break;
      }
      if (lst[m] < qn) a = m + 1;
      else b = m - 1;
    }
    if (hit >= 0) {
      const uint32_t npf = qn | (pf & (REC_BOND | REC_ACTIVE));
      recs[first + hit * rs] = make_uint4(npf, rf.y, rf.z, rf.w);
      carried[hit >> 5] |= 1u << (hit & 31);
    } else if ((pf & REC_BOND) && d.posq[cur][qn].w > 0) {
      // a bond may leave the list only with a partner that left the domain
      if (atomicCAS(&d.ctl->lost_i, -1, d.id[pc][p]) == -1) {
        const int4 qq = d.posq[cur][qn];
        const int dx = (int)((uint32_t)qq.x - (uint32_t)pq.x);
        const int dy = (int)((uint32_t)qq.y - (uint32_t)pq.y);
        const int dz = (int)((uint32_t)qq.z - (uint32_t)pq.z);
        d.ctl->lost_j = d.id[pc][qn];
        d.ctl->lost_d2 = (unsigned long long)((long long)dx * dx) + (unsigned long long)((long long)dy * dy) +
                         (unsigned long long)((long long)dz * dz);
        const unsigned long long S = (unsigned long long)(unsigned)pq.w + (unsigned)qq.w +
                                     (unsigned)d.sp[d.sample[pc][p]].skin_q;
        d.ctl->lost_S2 = S * S;
      }
      latch(d.ctl, ST_BOND_LOST);
    }
  }
  // entries with a state (bonds, touching pairs, springs) first, in partner
  // order, then the candidates without one: the force kernel's warps then
  // meet the stateless entries, which need no contact law, in the same
  // iterations (a list's order is free once the carry above has used its
  // sort by partner)
  uint32_t ns = 0;
  for (uint32_t j = 0; j < n; ++j) {
    if (!((carried[j >> 5] >> (j & 31)) & 1u)) continue;
    if (ns != j) recs[first + ns * rs] = recs[first + j * rs];
    ++ns;
  }
  if (ns == 0 || ns == n) return;
  for (uint32_t j = 0; j < n; ++j)
    if (!((carried[j >> 5] >> (j & 31)) & 1u)) recs[first + (ns++) * rs] = make_uint4(lst[j], 0u, 0u, 0u);
}

// FP64: sort each candidate list by partner.  A sphere owns the pairs with
// its higher-index partners: their records (zero history) are packed so that
// the records of a segment of ppw consecutive spheres (one warp of the force
// kernel) are contiguous.  Its lower-index partners are kept for k_rb_carry.
template <bool MIXED>
__global__ void k_rb_lists_half(Dev d) {
  if (!d.ctl->rebuild) return;
  const int nxt = d.ctl->cur ^ 1;
  const int rn = d.ctl->rec_cur ^ 1;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;  // grid covers Npad exactly
  const int lane = threadIdx.x & 31;
  const int Npad = d.Npad, cap = d.cap;
  if (p - lane >= Npad) return;  // whole warps only (Npad is a multiple of 256)
  const bool valid = p < d.N;
  uint32_t count = valid ? d.cand_n[p] : 0u;
  if (count > (uint32_t)cap) latch(d.ctl, ST_CAPACITY);
  unsigned mx = count, sum = count;
#pragma unroll
  for (int k = 16; k >= 1; k >>= 1) {
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, k));
    sum += __shfl_xor_sync(0xffffffffu, sum, k);
  }
  if (lane == 0 && sum) {
    atomicMax(&d.ctl->max_cand_next, (int)mx);
    atomicAdd((unsigned long long*)&d.ctl->cand_total_next, (unsigned long long)sum);
  }
  const uint32_t n = count < (uint32_t)cap ? count : (uint32_t)cap;
  // insertion sort by partner index (lists are short; sizes vary with the PSD)
  uint32_t lst[CGDEM_MAX_NEIGHBORS];
  uint32_t nl = 0;  // lower-index partners come first
  if (valid) {
    for (uint32_t j = 0; j < n; ++j) {
      const uint32_t v = d.cand_tmp[(size_t)j * Npad + p];
      uint32_t i = j;
      while (i > 0 && lst[i - 1] > v) {
        lst[i] = lst[i - 1];
        --i;
      }
      lst[i] = v;
    }
    while (nl < n && lst[nl] < (uint32_t)p) ++nl;
  }
  const uint32_t nu = n - nl;
  const int P = d.ppw, sub = lane & (P - 1);
  uint32_t incl = nu;
#pragma unroll
  for (int k = 1; k < 32; k <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, k, P);
    if (k < P && sub >= k) incl += y;
  }
  const uint32_t seg = (uint32_t)(p - sub) * (uint32_t)cap;
  const uint32_t first = seg + incl - nu;
  d.roff[rn][p] = first;
  d.cnt[rn][p] = nu;
  d.inc_n[p] = nl;
  if (sub == 0) d.seg_wait[p / P] = (uint32_t)(p / P);  // lowered by k_rb_carry
  if (!valid) return;
  d.posq_ref[p] = d.posq[nxt][p];
  for (uint32_t j = 0; j < nu; ++j) {
    if (MIXED) {
      reinterpret_cast<uint4*>(d.rec[rn])[first + j] = make_uint4(lst[nl + j], 0u, 0u, 0u);
    } else {
      RecD* rr = reinterpret_cast<RecD*>(d.rec[rn]) + first + j;
      *reinterpret_cast<int4*>(rr) = make_int4((int)lst[nl + j], 0, 0, 0);
      *(reinterpret_cast<double2*>(rr) + 1) = make_double2(0.0, 0.0);
    }
    d.rslot[first + j] = 0xffffffffu;  // set by k_rb_carry from the partner's side
  }
  for (uint32_t k = 0; k < nl; ++k) d.inc[(size_t)k * Npad + p] = lst[k];
}

// Record index of the pair (owner, partner) in list buffer b, or UINT_MAX.
// Lists are sorted by partner; only the partner bits of the first word are
// read (another thread may be rewriting the flags of the same word).
__device__ __forceinline__ uint32_t find_record(const Dev& d, int b, uint32_t owner, uint32_t partner) {
  const uint32_t base = d.roff[b][owner];
  int lo = 0, hi = (int)d.cnt[b][owner] - 1;
  while (lo <= hi) {
    const int m = (lo + hi) >> 1;
    const size_t idx = (size_t)base + (size_t)m * d.rstride;
    const uint32_t pf = d.mixed ? reinterpret_cast<const uint4*>(d.rec[b])[idx].x
                                : reinterpret_cast<const RecD*>(d.rec[b])[idx].pf;
    const uint32_t q = pf & REC_IDX;
    if (q == partner) return (uint32_t)idx;
    if (q < partner) lo = m + 1;
    else hi = m - 1;
  }
  return 0xffffffffu;
}

// FP64, after k_rb_lists_half: (1) the record of each pair a lower-index partner owns
// learns its slot in this sphere's inbox; (2) the contact history of the old
// lists moves to the pair's record in the new lists, negated when the
// pair's owner changed (the other sphere's tangential spring is the
// opposite vector, Eq. 4).
template <bool MIXED>
__global__ void k_rb_carry(Dev d) {
  if (!d.ctl->rebuild) return;
  const int nxt = d.ctl->cur ^ 1;
  const int pn = d.ctl->pcur ^ 1;
  const int rc = d.ctl->rec_cur, rn = rc ^ 1;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= d.N) return;
  const size_t Npad = (size_t)d.Npad;
  const uint32_t nl = d.inc_n[p];
  // the force kernel's warp of this sphere waits for the warp owning its
  // lowest partner (the list is sorted)
  if (nl) atomicMin(&d.seg_wait[p / d.ppw], d.inc[p] / (uint32_t)d.ppw);
  for (uint32_t k = 0; k < nl; ++k) {
    const uint32_t q = d.inc[k * Npad + p];
    const uint32_t e = find_record(d, rn, q, (uint32_t)p);
    if (e == 0xffffffffu) {  // the candidate relation lost its symmetry: a list overflowed
      latch(d.ctl, ST_CAPACITY);
      d.inc_n[p] = k;
      break;
    }
    d.rslot[e] = k;
  }
  const int4 pq = d.posq[nxt][p];
  if (pq.w <= 0) return;  // a sphere that left the domain drops its pairs
  const uint32_t o = d.perm[p];
  const uint32_t nold = d.cnt[rc][o];
  const uint32_t oldfirst = d.roff[rc][o];
  for (uint32_t k = 0; k < nold; ++k) {
    const size_t oidx = (size_t)oldfirst + (size_t)k * d.rstride;
    uint32_t pf;
    bool nz;
    uint4 rf = make_uint4(0, 0, 0, 0);
    int4 h0 = make_int4(0, 0, 0, 0);
    double2 h1 = make_double2(0, 0);
    if (MIXED) {
      rf = reinterpret_cast<const uint4*>(d.rec[rc])[oidx];
      pf = rf.x;
      nz = (rf.y | rf.z | rf.w) != 0u;
    } else {
      const RecD* rr = reinterpret_cast<const RecD*>(d.rec[rc]) + oidx;
      h0 = *reinterpret_cast<const int4*>(rr);
      h1 = *(reinterpret_cast<const double2*>(rr) + 1);
      pf = (uint32_t)h0.x;
      nz = (h0.z | h0.w) != 0 || h1.x != 0.0 || h1.y != 0.0;
    }
    if (!(pf & (REC_BOND | REC_ACTIVE)) && !nz) continue;
    const uint32_t qn = d.inv_perm[pf & REC_IDX];
    const bool mine = (uint32_t)p < qn;
    const uint32_t owner = mine ? (uint32_t)p : qn, partner = mine ? qn : (uint32_t)p;
    const uint32_t e = find_record(d, rn, owner, partner);
    if (e != 0xffffffffu) {
      const uint32_t npf = partner | (pf & (REC_BOND | REC_ACTIVE));
      if (MIXED) {
        uint4 w = make_uint4(npf, rf.y, rf.z, rf.w);
        if (!mine) {
          w.y = __float_as_uint(-__uint_as_float(rf.y));
          w.z = __float_as_uint(-__uint_as_float(rf.z));
          w.w = __float_as_uint(-__uint_as_float(rf.w));
        }
        reinterpret_cast<uint4*>(d.rec[rn])[e] = w;
      } else {
        double hx = __hiloint2double(h0.w, h0.z);
        double2 hyz = h1;
        if (!mine) {
          hx = -hx;
          hyz = make_double2(-h1.x, -h1.y);
        }
        RecD* rr = reinterpret_cast<RecD*>(d.rec[rn]) + e;
        *reinterpret_cast<int4*>(rr) = make_int4((int)npf, 0, __double2loint(hx), __double2hiint(hx));
        *(reinterpret_cast<double2*>(rr) + 1) = hyz;
      }
    } else if ((pf & REC_BOND) && d.posq[nxt][qn].w > 0) {
      // a bond may leave the list only with a partner that left the domain
      if (atomicCAS(&d.ctl->lost_i, -1, d.id[pn][p]) == -1) {
        const int4 qq = d.posq[nxt][qn];
        const int dx = (int)((uint32_t)qq.x - (uint32_t)pq.x);
        const int dy = (int)((uint32_t)qq.y - (uint32_t)pq.y);
        const int dz = (int)((uint32_t)qq.z - (uint32_t)pq.z);
        d.ctl->lost_j = d.id[pn][qn];
        d.ctl->lost_d2 = (unsigned long long)((long long)dx * dx) + (unsigned long long)((long long)dy * dy) +
                         (unsigned long long)((long long)dz * dz);
        const unsigned long long S = (unsigned long long)(unsigned)pq.w + (unsigned)qq.w +
                                     (unsigned)d.sp[d.sample[pn][p]].skin_q;
        d.ctl->lost_S2 = S * S;
      }
      latch(d.ctl, ST_BOND_LOST);
    }
  }
}

__global__ void k_rb_finish(Dev d) {
  Ctl* c = d.ctl;
  if (!c->rebuild) return;
  if (!d.mixed) {  // mixed: k_rb_permute2 wrote the state back into the current buffers
    c->cur ^= 1;
    c->pcur ^= 1;
  }
  c->rec_cur ^= 1;
  c->rebuild = 0;
  c->max_cand = c->max_cand_next;
  c->cand_total = c->cand_total_next;
  c->max_cand_next = 0;
  c->cand_total_next = 0;
  c->rebuilds += 1;
  for (int s = 0; s < d.n_samples; ++s) d.dmax2[s] = 0u;
}

__global__ void k_set_rebuild(Dev d) {
  d.ctl->rebuild = 1;
}

// Bond every candidate pair that touches (d^2 < (Ri+Rj)^2 in IEEE double).
__global__ void k_bond_touching(Dev d) {
  const int cur = d.ctl->cur, pc = d.ctl->pcur, rc = d.ctl->rec_cur;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= d.N) return;
  const double4 P = d.pos[cur][p];
  if (!(P.w > 0.0)) return;
  const SampleDev& S = d.sp[d.sample[pc][p]];
  const uint32_t n = d.cnt[rc][p];
  for (uint32_t k = 0; k < n; ++k) {
    const size_t idx = (size_t)d.roff[rc][p] + (size_t)k * d.rstride;
    uint32_t* pfp = d.mixed ? &reinterpret_cast<uint4*>(d.rec[rc])[idx].x
                            : &reinterpret_cast<RecD*>(d.rec[rc])[idx].pf;
    const uint32_t q = *pfp & REC_IDX;
    const double4 Q = d.pos[cur][q];
    if (!(Q.w > 0.0)) continue;
    double d2, Sd;
    exact_geometry(S, P, Q, &d2, &Sd);
    if (d2 < __dmul_rn(Sd, Sd)) *pfp |= REC_BOND;
  }
}

// ---------------------------------------------------------------------------
// porosity (void-fraction) scatter, fixed point
// ---------------------------------------------------------------------------

__global__ void k_vf_zero(Dev d, int which_offset) {
  const int b = (d.ctl->vf_cur + which_offset) % 3;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < d.Cf_total; c += gridDim.x * blockDim.x)
    d.vf[b][c] = 0ull;
}

// Equal-volume cube (side (pi/6)^(1/3) d) spread over the cells it overlaps.
__device__ void scatter_cube(const SampleDev& S, double4 P, unsigned long long* out) {
  const double side = __dmul_rn(__dmul_rn(2.0, fabs(P.w)), 0.8059959770082348);
  const double p3[3] = {P.x, P.y, P.z};
  double lo[3], hi[3];
  int a0[3], a1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    lo[k] = __dsub_rn(p3[k], __dmul_rn(0.5, side));
    hi[k] = __dadd_rn(p3[k], __dmul_rn(0.5, side));
    double t0 = floor(__dmul_rn(__dsub_rn(lo[k], S.f_lo[k]), S.inv_hf[k]));
    double t1 = floor(__dmul_rn(__dsub_rn(hi[k], S.f_lo[k]), S.inv_hf[k]));
    // a diverged (non-finite or far-away) position must not drive the loops
    const double lim = 4.0 * (double)S.nf[k] + 4.0;
    if (!(t0 >= -lim && t0 <= lim) || !(t1 >= -lim && t1 <= lim) || t1 - t0 > (double)S.nf[k] + 2.0)
      return;
    a0[k] = (int)t0;
    a1[k] = (int)t1;
  }
  for (int az = a0[2]; az <= a1[2]; ++az)
    for (int ay = a0[1]; ay <= a1[1]; ++ay)
      for (int ax = a0[0]; ax <= a1[0]; ++ax) {
        const int a[3] = {ax, ay, az};
        double vol = 1.0;
        int c[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const double b0 = __dadd_rn(S.f_lo[k], __dmul_rn((double)a[k], S.hf[k]));
          const double b1 = __dadd_rn(S.f_lo[k], __dmul_rn((double)(a[k] + 1), S.hf[k]));
          double ov = __dsub_rn(fmin(hi[k], b1), fmax(lo[k], b0));
          if (ov < 0.0) ov = 0.0;
          vol = __dmul_rn(vol, ov);
          int ck = a[k];
          if (S.kind == CGDEM_PERIODIC_BOX) {
            ck %= S.nf[k];
            if (ck < 0) ck += S.nf[k];
          } else {
            if (ck < 0) ck = 0;
            if (ck > S.nf[k] - 1) ck = S.nf[k] - 1;
          }
          c[k] = ck;
        }
        if (vol <= 0.0) continue;
        const int cell = S.fcell_off + (c[2] * S.nf[1] + c[1]) * S.nf[0] + c[0];
        atomicAdd(&out[cell], (unsigned long long)__double2ll_rn(__dmul_rn(vol, S.inv_q)));
      }
}

// Scatter the quanta of all active particles into buffer (vf_cur + offset).
// Centroid mode uses the stored fluid cell; cube mode recomputes the parts.
__global__ void k_vf_scatter(Dev d, int which_offset) {
  const int cur = d.ctl->cur, pc = d.ctl->pcur;
  const int b = (d.ctl->vf_cur + which_offset) % 3;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= d.N) return;
  const double4 P = d.pos[cur][p];
  if (!(P.w > 0.0)) return;
  const SampleDev& S = d.sp[d.sample[pc][p]];
  if (S.vf_mode == 0)
    atomicAdd(&d.vf[b][d.fcell[pc][p]], d.vq[pc][p]);
  else
    scatter_cube(S, P, d.vf[b]);
}

// Cube-mode scatter for the fused step (positions already drifted into the
// other buffer by the force kernel; runs after it, before its bookkeeping).
__global__ void k_vf_scatter_cube_next(Dev d) {
  const int cur = d.ctl->cur;  // the state written by the last force kernel
  const int pc = d.ctl->pcur;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= d.N) return;
  const double4 P = d.pos[cur][p];
  if (!(P.w > 0.0)) return;
  const SampleDev& S = d.sp[d.sample[pc][p]];
  if (S.vf_mode == 1 && (d.ctl->step % S.couple_every) == 0) scatter_cube(S, P, d.vf[d.ctl->vf_cur]);
}

__global__ void k_vf_rotate(Dev d) { d.ctl->vf_cur = (d.ctl->vf_cur + 1) % 3; }

// ---------------------------------------------------------------------------
// velocity Verlet halves (API verbs)
// ---------------------------------------------------------------------------

__device__ __forceinline__ void write_shadows(Dev& d, int buf, int p, const SampleDev& S, double4 P,
                                              double4 V, double4 W) {
  int4 q = d.posq[buf][p];
  q.x = to_q(P.x, S.inv_dq);
  q.y = to_q(P.y, S.inv_dq);
  q.z = to_q(P.z, S.inv_dq);
  if (!(P.w > 0.0)) q.w = 0;
  d.posq[buf][p] = q;
  d.velf[buf][p] = make_float4((float)V.x, (float)V.y, (float)V.z, (float)fabs(P.w));
  d.omgf[buf][p] = make_float4((float)W.x, (float)W.y, (float)W.z, (float)(1.0 / V.w));
}

// half kick + drift (in place); optionally scatter quanta into vf_cur+1.
__global__ void k_kick_drift(Dev d, int couple) {
  const int cur = d.ctl->cur, pc = d.ctl->pcur;
  const int b = (d.ctl->vf_cur + 1) % 3;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  float disp2 = -1.f;  // squared displacement since the rebuild (fixed units)
  int s = 0;
  if (p < d.N) {
    double4 P = d.pos[cur][p];
    s = d.sample[pc][p];
    if (P.w > 0.0) {
      const SampleDev& S = d.sp[s];
      double4 V = d.vel[cur][p], W = d.omg[cur][p];
      const double4 F = d.F[p], Tq = d.T[p];
      const double h = S.half_dt;
      V.x += h * (F.x * V.w);
      V.y += h * (F.y * V.w);
      V.z += h * (F.z * V.w);
      W.x += h * (Tq.x * W.w);
      W.y += h * (Tq.y * W.w);
      W.z += h * (Tq.z * W.w);
      double x = P.x + S.dt * V.x, y = P.y + S.dt * V.y, z = P.z + S.dt * V.z;
      if (S.kind == CGDEM_PERIODIC_BOX) {
        if (x >= S.L[0]) x -= S.L[0]; else if (x < 0.0) x += S.L[0];
        if (y >= S.L[1]) y -= S.L[1]; else if (y < 0.0) y += S.L[1];
        if (z >= S.L[2]) z -= S.L[2]; else if (z < 0.0) z += S.L[2];
      }
      P.x = x;
      P.y = y;
      P.z = z;
      d.pos[cur][p] = P;
      d.vel[cur][p] = V;
      d.omg[cur][p] = W;
      write_shadows(d, cur, p, S, P, V, W);
      const int fc = fluid_cell_of(S, x, y, z);
      d.fcell[pc][p] = fc;
      const int4 qn = d.posq[cur][p];
      const int4 ref = d.posq_ref[p];
      const float ex = (float)(int)((uint32_t)qn.x - (uint32_t)ref.x);
      const float ey = (float)(int)((uint32_t)qn.y - (uint32_t)ref.y);
      const float ez = (float)(int)((uint32_t)qn.z - (uint32_t)ref.z);
      disp2 = ex * ex + ey * ey + ez * ez;
      if (couple && (d.ctl->step % S.couple_every) == 0) {
        if (S.vf_mode == 0) atomicAdd(&d.vf[b][fc], d.vq[pc][p]);
        else scatter_cube(S, P, d.vf[b]);
      }
    }
  }
  // per-sample maximum: one atomic per warp when the warp holds one sample
  const unsigned FULLM = 0xffffffffu;
  const int s0 = __shfl_sync(FULLM, s, 0);
  if (__all_sync(FULLM, p >= d.N || s == s0)) {
    float md = disp2;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) md = fmaxf(md, __shfl_xor_sync(FULLM, md, o));
    if ((threadIdx.x & 31) == 0 && md >= 0.f) atomicMax(&d.dmax2[s0], __float_as_uint(md));
  } else if (disp2 >= 0.f) {
    atomicMax(&d.dmax2[s], __float_as_uint(disp2));
  }
}

// After a drift: displacement bound, rebuild flag, porosity rotation.
__global__ void k_after_drift(Dev d, int couple) {
  Ctl* c = d.ctl;
  bool any = false;
  for (int s = 0; s < d.n_samples; ++s) {
    if (__uint_as_float(d.dmax2[s]) > d.sp[s].rebuild_q2) c->rebuild = 1;
    if ((c->step % d.sp[s].couple_every) == 0) any = true;
    if (d.sp[s].kind == CGDEM_CYLINDER) drift_boundaries(d.stage[s], d.sp[s].dt);  // with the grains
  }
  if (couple && any) {
    c->vf_cur = (c->vf_cur + 1) % 3;
    c->fl_pending = 1;  // the Darcy flow follows the new porosity
  }
}

// final half kick + outlet (in place), completes a step.
__global__ void k_kick_final(Dev d) {
  const int cur = d.ctl->cur, pc = d.ctl->pcur;
  const long long m = d.ctl->step + 1;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= d.N) return;
  double4 P = d.pos[cur][p];
  if (!(P.w > 0.0)) return;
  const SampleDev& S = d.sp[d.sample[pc][p]];
  double4 V = d.vel[cur][p], W = d.omg[cur][p];
  const double4 F = d.F[p], Tq = d.T[p];
  const double h = S.half_dt;
  V.x += h * (F.x * V.w);
  V.y += h * (F.y * V.w);
  V.z += h * (F.z * V.w);
  W.x += h * (Tq.x * W.w);
  W.y += h * (Tq.y * W.w);
  W.z += h * (Tq.z * W.w);
  if (S.kind == CGDEM_CYLINDER && P.z < -2.0 * P.w) {
    d.removed_step[d.id[pc][p]] = (int)m;
    record_produced(d, S, d.sample[pc][p], P.w);
    P.w = -P.w;
    d.pos[cur][p] = P;
  }
  d.vel[cur][p] = V;
  d.omg[cur][p] = W;
  write_shadows(d, cur, p, S, P, V, W);
}

__global__ void k_step_inc(Dev d) { d.ctl->step += 1; }

// ---------------------------------------------------------------------------
// initial state and readback
// ---------------------------------------------------------------------------

// staging layout (doubles): x[3N] v[3N] w[3N] R[N]
// The inputs of cgdem_init_particles: a radius outside (0, r_max] of its
// sample, or a non-finite sum of the nine state components (summed x, y, z
// of x, v, w in order), records the particle's index; the host reads the
// lowest of each.
__global__ void k_init_check(Dev d) {
  const double* st = d.staging;
  const long long N = d.N;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
       p += (long long)gridDim.x * blockDim.x) {
    int s = 0;
    while (s + 1 < d.n_samples && p >= d.sp[s + 1].first) ++s;
    const double R = st[9 * N + p];
    if (!(R > 0.0) || !(R <= d.sp[s].r_max)) atomicMin(&d.ctl->init_bad_r, p);
    double t = st[3 * p];
    t = __dadd_rn(t, st[3 * p + 1]);
    t = __dadd_rn(t, st[3 * p + 2]);
    for (int k = 1; k < 3; ++k) {
      const double* a = st + 3 * N * k + 3 * p;
      t = __dadd_rn(t, a[0]);
      t = __dadd_rn(t, a[1]);
      t = __dadd_rn(t, a[2]);
    }
    if (!isfinite(t)) atomicMin(&d.ctl->init_bad_f, p);
  }
}

__global__ void k_init_state(Dev d) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= d.N) return;
  const double* st = d.staging;
  const int N = d.N;
  int s = 0;
  while (s + 1 < d.n_samples && p >= d.sp[s + 1].first) ++s;
  const SampleDev& S = d.sp[s];
  const double R = st[9 * (size_t)N + p];
  const double c = 4.1887902047863905;
  const double m = S.rho * (c * R * R * R);
  const double I = 0.4 * m * R * R;
  double4 P = make_double4(st[3 * p], st[3 * p + 1], st[3 * p + 2], R);
  double4 V = make_double4(st[3 * N + 3 * p], st[3 * N + 3 * p + 1], st[3 * N + 3 * p + 2], 1.0 / m);
  double4 W = make_double4(st[6 * N + 3 * p], st[6 * N + 3 * p + 1], st[6 * N + 3 * p + 2], 1.0 / I);
  if (S.kind == CGDEM_PERIODIC_BOX) {
    // bring positions into [0, L)
    double* xs[3] = {&P.x, &P.y, &P.z};
    for (int k = 0; k < 3; ++k) {
      double v = *xs[k];
      if (v >= S.L[k] || v < 0.0) {
        v = fmod(v, S.L[k]);
        if (v < 0.0) v += S.L[k];
        if (v >= S.L[k]) v -= S.L[k];
      }
      *xs[k] = v;
    }
  }
  const int cur = 0;
  d.pos[cur][p] = P;
  d.vel[cur][p] = V;
  d.omg[cur][p] = W;
  d.posq[cur][p] = make_int4(0, 0, 0, (int)llrint(R * S.inv_dq));
  write_shadows(d, cur, p, S, P, V, W);
  d.F[p] = make_double4(0, 0, 0, 0);
  d.T[p] = make_double4(0, 0, 0, 0);
  d.id[cur][p] = p;
  d.sample[cur][p] = s;
  d.fcell[cur][p] = fluid_cell_of(S, P.x, P.y, P.z);
  d.vq[cur][p] = volume_quantum(R, S.inv_q);
  d.removed_step[p] = -1;
  d.cnt[0][p] = 0;
  d.cnt[1][p] = 0;
  if (d.clc[0]) {
    d.clc[0][p] = make_float2(1.0f, 1.0f);
    d.clc[1][p] = make_float2(1.0f, 1.0f);
  }
  for (int w = 0; w < CGDEM_WALLS; ++w) {
    if (d.mixed && d.wallhf[cur]) d.wallhf[cur][(size_t)w * d.Npad + p] = make_float4(0, 0, 0, 0);
    if (!d.mixed && d.wallh[cur]) d.wallh[cur][(size_t)w * d.Npad + p] = make_double4(0, 0, 0, 0);
  }
}

__global__ void k_init_ctl(Dev d) {
  Ctl* c = d.ctl;
  c->cur = 0;
  c->pcur = 0;
  c->rec_cur = 0;
  c->vf_cur = 0;
  c->rebuild = 1;
  c->step = 0;
  c->rebuilds = 0;
  c->status = 0;
  c->block_counter = 0;
  c->blk_next = 0;
  c->epoch = 0;
  c->max_cand = 0;
  c->max_cand_next = 0;
  c->cand_total = 0;
  c->cand_total_next = 0;
  c->coupled = 0;
  c->closure = 0;
  c->record = 0;
  c->lost_i = -1;
  c->lost_j = -1;
  c->lost_d2 = 0;
  c->lost_S2 = 0;
  c->fl_pending = 0;
  c->fl_done = 1;
  c->fl_it = -1;
  c->fl_iters = 0;
  c->fl_bar_count = 0u;
  c->fl_bar_gen = 0u;
  c->fl_abort = 0;
  for (int s = 0; s < d.n_samples; ++s) d.dmax2[s] = 0u;
}

// staging layout (doubles): x[3N] v[3N] w[3N] F[3N] T[3N], id order
__global__ void k_gather_state(Dev d) {
  const int cur = d.ctl->cur, pc = d.ctl->pcur;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= d.N) return;
  const int i = d.id[pc][p];
  const size_t N = d.N;
  double* st = d.staging;
  const double4 P = d.pos[cur][p], V = d.vel[cur][p], W = d.omg[cur][p], F = d.F[p], T = d.T[p];
  st[3 * i] = P.x; st[3 * i + 1] = P.y; st[3 * i + 2] = P.z;
  st[3 * N + 3 * i] = V.x; st[3 * N + 3 * i + 1] = V.y; st[3 * N + 3 * i + 2] = V.z;
  st[6 * N + 3 * i] = W.x; st[6 * N + 3 * i + 1] = W.y; st[6 * N + 3 * i + 2] = W.z;
  st[9 * N + 3 * i] = F.x; st[9 * N + 3 * i + 1] = F.y; st[9 * N + 3 * i + 2] = F.z;
  st[12 * N + 3 * i] = T.x; st[12 * N + 3 * i + 1] = T.y; st[12 * N + 3 * i + 2] = T.z;
}

// Active contacts as (id_i, id_j | bond << 31) with id_i < id_j.
__global__ void k_collect_contacts(Dev d, uint32_t* out, unsigned long long cap) {
  const int pc = d.ctl->pcur, rc = d.ctl->rec_cur;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= d.N) return;
  const uint32_t n = d.cnt[rc][p];
  const int ip = d.id[pc][p];
  for (uint32_t k = 0; k < n; ++k) {
    const size_t idx = (size_t)d.roff[rc][p] + (size_t)k * d.rstride;
    const uint32_t pf = d.mixed ? reinterpret_cast<const uint4*>(d.rec[rc])[idx].x
                                : reinterpret_cast<const RecD*>(d.rec[rc])[idx].pf;
    if (!(pf & REC_ACTIVE)) continue;
    const int iq = d.id[pc][pf & REC_IDX];
    if (d.mixed && ip >= iq) continue;  // mixed lists hold each pair twice, FP64 lists once
    const unsigned long long slot = atomicAdd(d.contact_n, 1ull);
    if (slot < cap) {
      out[2 * slot] = (uint32_t)min(ip, iq);
      out[2 * slot + 1] = (uint32_t)max(ip, iq) | ((pf & REC_BOND) ? 0x80000000u : 0u);
    }
  }
}

// Active contacts with their tangential springs: (id_i, id_j | bond << 31)
// with id_i < id_j, and the spring as seen from id_i (the force-on-i
// convention of Eq. 4): mixed lists hold each pair twice and the lower id's
// record is taken; an FP64 pair is held by its lower-index sphere, whose
// spring is negated when that sphere has the higher id.
__global__ void k_collect_springs(Dev d, uint32_t* out, double* xi, unsigned long long cap) {
  const int pc = d.ctl->pcur, rc = d.ctl->rec_cur;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= d.N) return;
  const uint32_t n = d.cnt[rc][p];
  const int ip = d.id[pc][p];
  for (uint32_t k = 0; k < n; ++k) {
    const size_t idx = (size_t)d.roff[rc][p] + (size_t)k * d.rstride;
    uint32_t pf;
    double sx, sy, sz;
    if (d.mixed) {
      const uint4 r = reinterpret_cast<const uint4*>(d.rec[rc])[idx];
      pf = r.x;
      sx = __uint_as_float(r.y);
      sy = __uint_as_float(r.z);
      sz = __uint_as_float(r.w);
    } else {
      const RecD& r = reinterpret_cast<const RecD*>(d.rec[rc])[idx];
      pf = r.pf;
      sx = r.x;
      sy = r.y;
      sz = r.z;
    }
    if (!(pf & REC_ACTIVE)) continue;
    const int iq = d.id[pc][pf & REC_IDX];
    if (d.mixed && ip >= iq) continue;
    const double sg = ip < iq ? 1.0 : -1.0;
    const unsigned long long slot = atomicAdd(d.contact_n, 1ull);
    if (slot < cap) {
      out[2 * slot] = (uint32_t)min(ip, iq);
      out[2 * slot + 1] = (uint32_t)max(ip, iq) | ((pf & REC_BOND) ? 0x80000000u : 0u);
      xi[3 * slot] = sg * sx;
      xi[3 * slot + 1] = sg * sy;
      xi[3 * slot + 2] = sg * sz;
    }
  }
}

// Per-sample diagnostics: partial sums per block (fixed order), then reduce.
constexpr int DIAG_BLOCKS = 128;
__global__ void k_diag_partial(Dev d, double* part) {
  extern __shared__ double sh[];  // [n_samples * 8]
  const int cur = d.ctl->cur, pc = d.ctl->pcur, rc = d.ctl->rec_cur;
  const int S8 = d.n_samples * 8;
  for (int i = threadIdx.x; i < S8; i += blockDim.x) sh[i] = 0.0;
  __syncthreads();
  const int per = (d.N + gridDim.x - 1) / gridDim.x;
  const int b0 = blockIdx.x * per, b1 = min(d.N, b0 + per);
  // one thread walks the chunk in order: deterministic sums
  if (threadIdx.x == 0) {
    for (int p = b0; p < b1; ++p) {
      const double4 P = d.pos[cur][p], V = d.vel[cur][p], W = d.omg[cur][p];
      const int s = d.sample[pc][p];
      double* o = sh + 8 * s;
      const double m = 1.0 / V.w, I = 1.0 / W.w;
      if (P.w > 0.0) {
        o[0] += 0.5 * m * (V.x * V.x + V.y * V.y + V.z * V.z);
        o[1] += 0.5 * I * (W.x * W.x + W.y * W.y + W.z * W.z);
        o[2] += m * V.x;
        o[3] += m * V.y;
        o[4] += m * V.z;
        o[6] += 1.0;
        const uint32_t n = d.cnt[rc][p];
        const int ip = d.id[pc][p];
        for (uint32_t k = 0; k < n; ++k) {
          const size_t idx = (size_t)d.roff[rc][p] + (size_t)k * d.rstride;
          const uint32_t pf = d.mixed ? reinterpret_cast<const uint4*>(d.rec[rc])[idx].x
                                      : reinterpret_cast<const RecD*>(d.rec[rc])[idx].pf;
          if ((pf & REC_BOND) && (pf & REC_ACTIVE) && (!d.mixed || ip < d.id[pc][pf & REC_IDX]))
            o[7] += 1.0;  // mixed lists hold each pair twice
        }
      } else {
        o[5] += m;
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < S8; i += blockDim.x) part[(size_t)blockIdx.x * S8 + i] = sh[i];
}

__global__ void k_diag_reduce(Dev d, const double* part, int nblocks) {
  const int S8 = d.n_samples * 8;
  for (int i = threadIdx.x; i < S8; i += blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < nblocks; ++b) acc += part[(size_t)b * S8 + i];
    d.diag[i] = acc;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline int nblk(int n, int b) { return (n + b - 1) / b; }

void launch_rebuild(const Dev& d, cudaStream_t s) {
  const int B = 256, G = nblk(d.N, B);
  if (G == 0) return;
  k_rb_bin<<<G, B, 0, s>>>(d);
  const int ntiles = (d.C_total + 1 + SCAN_TILE - 1) / SCAN_TILE;
  k_rb_scan_tiles<<<ntiles, SCAN_T, 0, s>>>(d, d.tile_sums);
  k_rb_scan_sums<<<1, 1024, 0, s>>>(d, d.tile_sums, ntiles);
  k_rb_scan_apply<<<ntiles, SCAN_T, 0, s>>>(d, d.tile_sums);
  k_rb_scatter<<<G, B, 0, s>>>(d);
  k_rb_rank<<<G, B, 0, s>>>(d);
  k_rb_permute<<<G, B, 0, s>>>(d);
  k_rb_ft_gather<<<G, B, 0, s>>>(d);
  if (!d.mixed) k_rb_ft_store<<<G, B, 0, s>>>(d);
  k_rb_pairs<<<G, B, 0, s>>>(d);
  k_rb_pairs_big<<<4 * 152, 256, 0, s>>>(d);
  const int Gp = nblk(d.Npad, B);
  if (d.mixed) {
    k_rb_sched<<<nblk(d.Npad, SCHED_TILE), SCHED_TILE, 0, s>>>(d);
    k_rb_permute2<<<G, B, 0, s>>>(d);
    k_rb_ft_store<<<G, B, 0, s>>>(d);
    k_rb_lists_full<<<Gp, B, 0, s>>>(d);
  } else {
    k_rb_lists_half<false><<<Gp, B, 0, s>>>(d);
    k_rb_carry<false><<<G, B, 0, s>>>(d);
  }
  k_rb_finish<<<1, 1, 0, s>>>(d);
}

void launch_set_rebuild(const Dev& d, cudaStream_t s) { k_set_rebuild<<<1, 1, 0, s>>>(d); }

// First step of a captured block of steps: its rebuild node's condition from
// the device flag (the later steps' conditions are set by the force kernel
// of the step before).
__global__ void k_rebuild_cond(Dev d, cudaGraphConditionalHandle h) {
  cudaGraphSetConditional(h, d.ctl->rebuild ? 1u : 0u);
}
void launch_rebuild_cond(const Dev& d, cudaGraphConditionalHandle h, cudaStream_t s) {
  k_rebuild_cond<<<1, 1, 0, s>>>(d, h);
}


void launch_bond_touching(const Dev& d, cudaStream_t s) {
  if (d.N) k_bond_touching<<<nblk(d.N, 256), 256, 0, s>>>(d);
}

void launch_couple(const Dev& d, cudaStream_t s) {
  const int Gc = nblk(d.Cf_total, 256);
  if (Gc) {
    k_vf_zero<<<Gc, 256, 0, s>>>(d, 0);
    k_vf_zero<<<Gc, 256, 0, s>>>(d, 1);
  }
  if (d.N) k_vf_scatter<<<nblk(d.N, 256), 256, 0, s>>>(d, 0);
}

void launch_kick_drift(const Dev& d, int couple, cudaStream_t s) {
  if (d.N) k_kick_drift<<<nblk(d.N, 256), 256, 0, s>>>(d, couple);
  k_after_drift<<<1, 1, 0, s>>>(d, couple);
  // the buffer after the (possibly rotated) current one must be zero
  const int Gc = nblk(d.Cf_total, 256);
  if (couple && Gc) k_vf_zero<<<Gc, 256, 0, s>>>(d, 1);
}

// Spring history of one wall cleared for the spheres of one sample.
__global__ void k_clear_wall_history(Dev d, int sample, int wall) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= d.N) return;
  const int pc = d.ctl->pcur;
  if (d.sample[pc][p] != sample) return;
  const size_t i = (size_t)wall * d.Npad + p;
  if (d.mixed && d.wallhf[pc]) d.wallhf[pc][i] = make_float4(0, 0, 0, 0);
  if (!d.mixed && d.wallh[pc]) d.wallh[pc][i] = make_double4(0, 0, 0, 0);
}

void launch_clear_wall_history(const Dev& d, int sample, int wall, cudaStream_t s) {
  if (d.N) k_clear_wall_history<<<nblk(d.N, 256), 256, 0, s>>>(d, sample, wall);
}

void launch_kick_final(const Dev& d, cudaStream_t s) {
  if (d.N) k_kick_final<<<nblk(d.N, 256), 256, 0, s>>>(d);
  k_step_inc<<<1, 1, 0, s>>>(d);
}

void launch_cube_after_mid(const Dev& d, cudaStream_t s) {
  if (d.N) k_vf_scatter_cube_next<<<nblk(d.N, 256), 256, 0, s>>>(d);
}

// ---------------------------------------------------------------------------
// learned closure: switch, reset of the corrections, recorded data by id
// ---------------------------------------------------------------------------

__global__ void k_closure_set(Dev d, int enable, int record) {
  if (enable >= 0) d.ctl->closure = enable;
  if (record >= 0) d.ctl->record = record;
}

__global__ void k_closure_reset(Dev d) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= d.N) return;
  d.clc[0][p] = make_float2(1.0f, 1.0f);
  d.clc[1][p] = make_float2(1.0f, 1.0f);
}

// recorded rows in particle-id order, into the staging buffer (floats)
__global__ void k_closure_gather(Dev d) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= d.N) return;
  const int i = d.id[d.ctl->pcur][p];
  float* out = reinterpret_cast<float*>(d.staging);
  const float* in = d.clrec + (size_t)p * CL_COLS;
#pragma unroll
  for (int k = 0; k < CL_COLS; ++k) out[(size_t)i * CL_COLS + k] = in[k];
}

void launch_closure_set(const Dev& d, int enable, int record, cudaStream_t s) {
  k_closure_set<<<1, 1, 0, s>>>(d, enable, record);
  if (enable >= 0 && d.N) k_closure_reset<<<nblk(d.N, 256), 256, 0, s>>>(d);
}

void launch_closure_gather(const Dev& d, cudaStream_t s) {
  if (d.N) k_closure_gather<<<nblk(d.N, 256), 256, 0, s>>>(d);
}

void launch_init_check(const Dev& d, cudaStream_t s) {
  const int g = nblk(d.N, 256);
  if (d.N) k_init_check<<<g < 152 * 8 ? g : 152 * 8, 256, 0, s>>>(d);
}

void launch_init(const Dev& d, cudaStream_t s) {
  k_init_ctl<<<1, 1, 0, s>>>(d);
  if (d.N) k_init_state<<<nblk(d.N, 256), 256, 0, s>>>(d);
}

void launch_gather_state(const Dev& d, cudaStream_t s) {
  if (d.N) k_gather_state<<<nblk(d.N, 256), 256, 0, s>>>(d);
}

void launch_collect_springs(const Dev& d, uint32_t* out, double* xi, unsigned long long cap, cudaStream_t s) {
  cudaMemsetAsync(d.contact_n, 0, sizeof(unsigned long long), s);
  if (d.N) k_collect_springs<<<nblk(d.N, 256), 256, 0, s>>>(d, out, xi, cap);
}

void launch_collect_contacts(const Dev& d, uint32_t* out, unsigned long long cap, cudaStream_t s) {
  cudaMemsetAsync(d.contact_n, 0, sizeof(unsigned long long), s);
  if (d.N) k_collect_contacts<<<nblk(d.N, 256), 256, 0, s>>>(d, out, cap);
}

void launch_diag(const Dev& d, double* part, cudaStream_t s) {
  const size_t sh = sizeof(double) * 8 * d.n_samples;
  k_diag_partial<<<DIAG_BLOCKS, 32, sh, s>>>(d, part);
  k_diag_reduce<<<1, 256, 0, s>>>(d, part, DIAG_BLOCKS);
}

}  // namespace cgdem
