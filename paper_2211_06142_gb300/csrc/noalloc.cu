// noalloc.cu -- cgdem_touching_pairs_noalloc: the cell-list pair search of
// the library as one call that allocates no device memory.
//
// Its scratch (cell of each sphere, cell counts and starts, the cell-sorted
// order) lives in one file-scope __device__ array of fixed size, which every
// GPU that loads the library holds until the process exits.  Every call
// reuses it: the counts are cleared at the start of each call, and calls
// whose GPU work overlaps (on different streams, or from different threads)
// race on it.
#include <cstdio>
#include <mutex>

#include "cgdem.h"

namespace {

constexpr int NA_MAX_N = CGDEM_NOALLOC_MAX_SPHERES;
constexpr int NA_MAX_CELLS = CGDEM_NOALLOC_MAX_CELLS;

struct NoallocScratch {
  unsigned cell_of[NA_MAX_N];
  unsigned slot[NA_MAX_N];
  unsigned order[NA_MAX_N];
  unsigned count[NA_MAX_CELLS + 1];
  unsigned start[NA_MAX_CELLS + 2];
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

struct Grid {
  double lo[3], L[3], inv_h[3];
  int nc[3];
  int periodic;
};

__device__ __forceinline__ int na_cell(const Grid& g, const double* x, int* c3) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double t = floor((x[k] - g.lo[k]) * g.inv_h[k]);
    if (!(t >= 0.0)) t = 0.0;  // also catches NaN
    if (!(t <= (double)(g.nc[k] - 1))) t = (double)(g.nc[k] - 1);
    c3[k] = (int)t;
  }
  return (c3[2] * g.nc[1] + c3[1]) * g.nc[0] + c3[0];
}

__global__ void na_clear(NoallocScratch* s, int ncells, unsigned long long* count) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= ncells; c += gridDim.x * blockDim.x)
    s->count[c] = 0u;
  if (blockIdx.x == 0 && threadIdx.x == 0) *count = 0ull;
}

__global__ void na_bin(NoallocScratch* s, Grid g, const double* x, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c3[3];
  const unsigned c = (unsigned)na_cell(g, x + 3 * (size_t)i, c3);
  s->cell_of[i] = c;
  s->slot[i] = atomicAdd(&s->count[c], 1u);
}

// one block: exclusive scan of the counts into starts
__global__ void __launch_bounds__(1024) na_scan(NoallocScratch* s, int ncells) {
  __shared__ unsigned ws[32];
  __shared__ unsigned carry;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0u;
  __syncthreads();
  for (int b0 = 0; b0 < ncells; b0 += 1024) {
    const int i = b0 + threadIdx.x;
    const unsigned v = i < ncells ? s->count[i] : 0u;
    unsigned incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) ws[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      unsigned w = ws[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      ws[lane] = w;
    }
    __syncthreads();
    const unsigned before = (wid > 0 ? ws[wid - 1] : 0u) + carry;
    if (i < ncells) s->start[i] = before + incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry = before + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) s->start[ncells] = carry;
}

__global__ void na_scatter(NoallocScratch* s, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  s->order[s->start[s->cell_of[i]] + s->slot[i]] = (unsigned)i;
}

// Pairs i < j with d^2 < (Ri + Rj + skin)^2, the squared distance summed
// x, y, z in IEEE double without contraction, minimum image when periodic.
__global__ void na_pairs(const NoallocScratch* s, Grid g, const double* x, const double* R, int n,
                         double skin, int* pairs, long long cap, unsigned long long* count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double xi[3] = {x[3 * (size_t)i], x[3 * (size_t)i + 1], x[3 * (size_t)i + 2]};
  const double Ri = R[i];
  int c3[3];
  na_cell(g, xi, c3);
  int lists[3][3], nl[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    nl[k] = 0;
    if (g.periodic && g.nc[k] < 3) {
      for (int a = 0; a < g.nc[k]; ++a) lists[k][nl[k]++] = a;
    } else {
      for (int off = -1; off <= 1; ++off) {
        int a = c3[k] + off;
        if (g.periodic) a = (a + g.nc[k]) % g.nc[k];
        else if (a < 0 || a >= g.nc[k]) continue;
        lists[k][nl[k]++] = a;
      }
    }
  }
  for (int iz = 0; iz < nl[2]; ++iz)
    for (int iy = 0; iy < nl[1]; ++iy)
      for (int ix = 0; ix < nl[0]; ++ix) {
        const int c = (lists[2][iz] * g.nc[1] + lists[1][iy]) * g.nc[0] + lists[0][ix];
        for (unsigned t = s->start[c]; t < s->start[c + 1]; ++t) {
          const int j = (int)s->order[t];
          if (j <= i) continue;
          double d[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            double v = __dsub_rn(x[3 * (size_t)j + k], xi[k]);
            if (g.periodic) {
              const double h = 0.5 * g.L[k];
              if (v > h) v = __dsub_rn(v, g.L[k]);
              else if (v < -h) v = __dadd_rn(v, g.L[k]);
            }
            d[k] = v;
          }
          const double d2 =
              __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
          const double S = __dadd_rn(__dadd_rn(Ri, R[j]), skin);
          if (d2 < __dmul_rn(S, S)) {
            const unsigned long long k = atomicAdd(count, 1ull);
            if ((long long)k < cap) {
              pairs[2 * k] = i;
              pairs[2 * k + 1] = j;
            }
          }
        }
      }
}

std::mutex g_addr_mu;
void* g_addr[64] = {nullptr};

}  // namespace

extern "C" int cgdem_touching_pairs_noalloc(const double* x, const double* R, int64_t n,
                                            const double* box_lo, const double* box_hi,
                                            int periodic, double r_max, double skin,
                                            int32_t* pairs, int64_t cap,
                                            unsigned long long* count, void* stream) {
  if (!x || !R || !box_lo || !box_hi || !count || (!pairs && cap > 0) || n < 0 || cap < 0 ||
      !(r_max > 0) || !(skin >= 0)) {
    fprintf(stderr, "cgdem_touching_pairs_noalloc: invalid argument\n");
    return CGDEM_E_INVALID;
  }
  if (n > NA_MAX_N) {
    fprintf(stderr, "cgdem_touching_pairs_noalloc: %lld spheres exceed the fixed scratch limit %d\n",
            (long long)n, NA_MAX_N);
    return CGDEM_E_CAPACITY;
  }
  Grid g;
  const double h = 2.0 * r_max + skin;
  long long ncells = 1;
  for (int k = 0; k < 3; ++k) {
    g.lo[k] = box_lo[k];
    g.L[k] = box_hi[k] - box_lo[k];
    if (!(g.L[k] > 0)) {
      fprintf(stderr, "cgdem_touching_pairs_noalloc: empty box\n");
      return CGDEM_E_INVALID;
    }
    // cells a little wider than h: the cell coordinate (x - lo) * inv_h is
    // rounded, and a pair closer than h must never land two cells apart
    double nd = floor(g.L[k] / (h * (1.0 + 1e-9)));
    if (!(nd >= 1.0)) nd = 1.0;
    if (nd > (double)NA_MAX_CELLS) nd = (double)NA_MAX_CELLS;
    const int nc = (int)nd;
    g.nc[k] = nc;
    g.inv_h[k] = nc / g.L[k];
    ncells *= nc;
  }
  if (periodic && !(h < 0.5 * g.L[0] && h < 0.5 * g.L[1] && h < 0.5 * g.L[2])) {
    fprintf(stderr, "cgdem_touching_pairs_noalloc: periodic box smaller than 2 (2 r_max + skin)\n");
    return CGDEM_E_INVALID;
  }
  if (ncells > NA_MAX_CELLS) {
    fprintf(stderr, "cgdem_touching_pairs_noalloc: %lld cells exceed the fixed scratch limit %d; "
            "use a larger r_max or a smaller box\n", ncells, NA_MAX_CELLS);
    return CGDEM_E_CAPACITY;
  }
  g.periodic = periodic ? 1 : 0;
  // set-up, once per device: the device address of the scratch array
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    fprintf(stderr, "cgdem_touching_pairs_noalloc: no current device (%s)\n", cudaGetErrorString(e));
    return CGDEM_E_CUDA;
  }
  void* addr = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
      e = cudaGetSymbolAddress(&g_addr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_addr[dev] = nullptr;
        fprintf(stderr, "cgdem_touching_pairs_noalloc: cudaGetSymbolAddress failed: %s\n",
                cudaGetErrorString(e));
        return CGDEM_E_CUDA;
      }
    }
    addr = g_addr[dev];
  }
  NoallocScratch* s = static_cast<NoallocScratch*>(addr);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int nc = (int)ncells;
  na_clear<<<(nc + 256) / 256, 256, 0, st>>>(s, nc, count);
  if (n > 0) {
    const int G = (int)((n + 255) / 256);
    na_bin<<<G, 256, 0, st>>>(s, g, x, (int)n);
    na_scan<<<1, 1024, 0, st>>>(s, nc);
    na_scatter<<<G, 256, 0, st>>>(s, (int)n);
    na_pairs<<<G, 256, 0, st>>>(s, g, x, R, (int)n, skin, pairs, cap, count);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "cgdem_touching_pairs_noalloc: launch failed: %s\n", cudaGetErrorString(e));
    return CGDEM_E_CUDA;
  }
  return CGDEM_OK;
}
