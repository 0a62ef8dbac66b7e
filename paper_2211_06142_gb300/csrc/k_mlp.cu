// k_mlp.cu -- training and batch inference of the learned-closure network on
// the fifth-generation tensor cores (tcgen05, BF16 operands, FP32
// accumulators in tensor memory).
//
// One CTA of 128 threads owns one SM (170 KB of shared memory, all 512 TMEM
// columns) and walks tiles of 128 samples; thread t owns sample row t of
// the tile.  Per tile:
//   forward   Z_l = A_(l-1) W_l^T (M = 128, K = 16 or 64, N = 64 or 16),
//             epilogue adds b_l and applies SiLU, writes A_l in BF16 as the
//             next product's A tile and, when training, transposed (sample
//             index along K) for the weight gradient;
//   backward  dZ_4 = (o - y) m / B; dA_(l-1) = dZ_l W_l (M = 128),
//             dZ_(l-1) = dA_(l-1) silu'(Z_(l-1)); the weight gradients
//             dW_l = dZ_l^T A_(l-1) accumulate over all of the CTA's tiles in
//             TMEM (M = 128 rows of output units, K = 128 samples per tile,
//             N = inputs of the layer plus one column of ones that yields the
//             bias gradient of the hidden layers in the same product).
// Per-CTA gradient sums go to a workspace; k_mlp_adam adds them in a fixed
// order (deterministic) and applies Adam.
#include <cstdio>

#include "cgdem.h"
#include "cgdem_internal.cuh"
#include "closure.cuh"
#include "tc05.cuh"

namespace {

using namespace tc05;
using namespace closure;

constexpr int TROWS = 128;
constexpr int MAX_GRID = 256;

// shared-memory tiles (byte offsets from a 1024-aligned base)
constexpr uint32_t S_W1 = 0;                  // W1   [64 x 16]
constexpr uint32_t S_W2 = S_W1 + 2048;        // W2   [64 x 64]
constexpr uint32_t S_W3 = S_W2 + 8192;        // W3   [64 x 64]
constexpr uint32_t S_W4 = S_W3 + 8192;        // W4   [16 x 64] (rows >= 2 zero)
constexpr uint32_t S_W2T = S_W4 + 2048;       // W2^T [64 x 64]
constexpr uint32_t S_W3T = S_W2T + 8192;      // W3^T [64 x 64]
constexpr uint32_t S_W4T = S_W3T + 8192;      // W4^T [64 x 16] (columns >= 2 zero)
constexpr uint32_t S_A0 = S_W4T + 2048;       // x_hat        [128 x 16]
constexpr uint32_t S_AH = S_A0 + 4096;        // h_l          [128 x 64]
constexpr uint32_t S_X0T = S_AH + 16384;      // x_hat^T, ones row 5        [16 x 128]
constexpr uint32_t S_X1T = S_X0T + 4096;      // h_1^T, ones row 64         [80 x 128]
constexpr uint32_t S_X2T = S_X1T + 20480;     // h_2^T                      [80 x 128]
constexpr uint32_t S_X3T = S_X2T + 20480;     // h_3^T                      [80 x 128]
constexpr uint32_t S_DZ = S_X3T + 20480;      // dZ_l rows    [128 x 64] (dZ_4: [128 x 16])
constexpr uint32_t S_DZT = S_DZ + 16384;      // dZ_l^T rows 0-63, dZ_4^T rows 64-65 [128 x 128]
constexpr uint32_t S_INF_END = S_AH + 16384;  // inference needs the tiles up to here
constexpr uint32_t S_END = S_DZT + 32768;

// TMEM columns
constexpr uint32_t C_Z1 = 0, C_Z2 = 64, C_Z3 = 128, C_O = 192, C_DA = 192;
constexpr uint32_t C_DW4 = 256, C_DW2 = 320, C_DW3 = 416, C_DW1 = 496;

// logistic function with the hardware exponential and reciprocal (a few ulp
// in FP32, far below the BF16 rounding of the activations; 0 where the
// exponential overflows)
__device__ __forceinline__ float sigm(float z) { return __fdividef(1.0f, 1.0f + __expf(-z)); }

__device__ __forceinline__ void st_bf16(uint8_t* sm, uint32_t off, float v) {
  *reinterpret_cast<unsigned short*>(sm + off) = bf16_bits(v);
}

// all threads wait for the MMA group committed on mbar; false on timeout
__device__ __forceinline__ bool wait_mma(uint64_t* mbar, uint32_t& phase) {
  const bool ok = mbar_wait(mbar, phase);
  phase ^= 1u;
  const int bad = __syncthreads_or(!ok);
  fence_after_sync();
  return bad == 0;
}

// make this thread's shared-memory tile writes visible to the tensor core
// and order them before the MMA issued after the barrier
__device__ __forceinline__ void publish_tiles() {
  fence_smem_to_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
}

__device__ void build_weight_tiles(const float* __restrict__ th, uint8_t* sm, bool train) {
  for (int e = threadIdx.x; e < 64 * 16; e += blockDim.x) {  // W1 [i][j<5]
    const int i = e >> 4, j = e & 15;
    st_bf16(sm, S_W1 + tile_off(i, j, 16), j < N_IN ? th[OFF_W1 + i * N_IN + j] : 0.0f);
  }
  for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
    const int i = e >> 6, j = e & 63;
    const float w2 = th[OFF_W2 + e], w3 = th[OFF_W3 + e];
    st_bf16(sm, S_W2 + tile_off(i, j, 64), w2);
    st_bf16(sm, S_W3 + tile_off(i, j, 64), w3);
    if (train) {
      st_bf16(sm, S_W2T + tile_off(j, i, 64), w2);
      st_bf16(sm, S_W3T + tile_off(j, i, 64), w3);
    }
  }
  for (int e = threadIdx.x; e < 16 * 64; e += blockDim.x) {  // W4 [k<2][j]
    const int k = e >> 6, j = e & 63;
    const float w = k < N_OUT ? th[OFF_W4 + k * N_H + j] : 0.0f;
    st_bf16(sm, S_W4 + tile_off(k, j, 64), w);
    if (train) st_bf16(sm, S_W4T + tile_off(j, k, 16), w);
  }
}

// constant parts of the training tiles: ones rows, zero rows
__device__ void init_train_tiles(uint8_t* sm) {
  for (int e = threadIdx.x; e < 16 * 128; e += blockDim.x) {
    const int r = e >> 7, b = e & 127;
    if (r >= N_IN) st_bf16(sm, S_X0T + tile_off(r, b, 128), r == N_IN ? 1.0f : 0.0f);
  }
  for (int e = threadIdx.x; e < 16 * 128; e += blockDim.x) {
    const int r = 64 + (e >> 7), b = e & 127;
    const float v = r == 64 ? 1.0f : 0.0f;
    st_bf16(sm, S_X1T + tile_off(r, b, 128), v);
    st_bf16(sm, S_X2T + tile_off(r, b, 128), v);
    st_bf16(sm, S_X3T + tile_off(r, b, 128), v);
  }
  for (int e = threadIdx.x; e < 32768 / 16; e += blockDim.x)
    reinterpret_cast<uint4*>(sm + S_DZT)[e] = make_uint4(0u, 0u, 0u, 0u);
}

// hidden-layer epilogue: h = silu(z + b) written as the next A tile and,
// when training, into the transposed tile at column `row`
__device__ __forceinline__ void hidden_epilogue(uint32_t tb, uint32_t col, const float* bias, uint8_t* sm,
                                                uint32_t s_xt, bool train) {
  const int row = threadIdx.x, warp = row >> 5;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float z[16];
    tmem_ld16(taddr(tb, 32u * warp, col + 16u * c), z);
    float h[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float zz = z[j] + bias[16 * c + j];
      h[j] = zz * sigm(zz);
    }
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      uint4 v;
      v.x = pack_bf16x2(h[8 * half + 0], h[8 * half + 1]);
      v.y = pack_bf16x2(h[8 * half + 2], h[8 * half + 3]);
      v.z = pack_bf16x2(h[8 * half + 4], h[8 * half + 5]);
      v.w = pack_bf16x2(h[8 * half + 6], h[8 * half + 7]);
      *reinterpret_cast<uint4*>(sm + S_AH + tile_off(row, 16 * c + 8 * half, 64)) = v;
    }
    if (train) {
#pragma unroll
      for (int j = 0; j < 16; ++j) st_bf16(sm, s_xt + tile_off(16 * c + j, row, 128), h[j]);
    }
  }
}

// backward epilogue of a hidden layer: dz = dA * silu'(z + b); writes the dZ
// row tile (when another dA product follows) and the transposed dZ^T rows
__device__ __forceinline__ void backward_epilogue(uint32_t tb, uint32_t col_z, const float* bias, uint8_t* sm,
                                                  bool write_rows) {
  const int row = threadIdx.x, warp = row >> 5;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float da[16], z[16];
    tmem_ld16(taddr(tb, 32u * warp, C_DA + 16u * c), da);
    tmem_ld16(taddr(tb, 32u * warp, col_z + 16u * c), z);
    float dz[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float zz = z[j] + bias[16 * c + j];
      const float s = sigm(zz);
      dz[j] = da[j] * (s * (1.0f + zz * (1.0f - s)));
    }
    if (write_rows) {
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        uint4 v;
        v.x = pack_bf16x2(dz[8 * half + 0], dz[8 * half + 1]);
        v.y = pack_bf16x2(dz[8 * half + 2], dz[8 * half + 3]);
        v.z = pack_bf16x2(dz[8 * half + 4], dz[8 * half + 5]);
        v.w = pack_bf16x2(dz[8 * half + 6], dz[8 * half + 7]);
        *reinterpret_cast<uint4*>(sm + S_DZ + tile_off(row, 16 * c + 8 * half, 64)) = v;
      }
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) st_bf16(sm, S_DZT + tile_off(16 * c + j, row, 128), dz[j]);
  }
}

template <bool TRAIN>
__global__ void __launch_bounds__(TROWS, 1)
    k_mlp(const float* __restrict__ theta, const float* __restrict__ X, const float* __restrict__ Y,
          const float* __restrict__ Mk, int n, float inv_n, float* __restrict__ out, float* __restrict__ part,
          int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tbase_s;
  __shared__ float bias_s[3][N_H];
  __shared__ float red_s[4][3];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sraw = smem_u32(smem_raw);
  const uint32_t s0 = (sraw + 1023u) & ~1023u;
  uint8_t* sm = smem_raw + (s0 - sraw);
  constexpr uint32_t NCOLS = TRAIN ? 512u : 256u;

  build_weight_tiles(theta, sm, TRAIN);
  if (TRAIN) init_train_tiles(sm);
  for (int e = tid; e < 3 * N_H; e += TROWS) {
    const int l = e / N_H, j = e % N_H;
    bias_s[l][j] = theta[(l == 0 ? OFF_B1 : l == 1 ? OFF_B2 : OFF_B3) + j];
  }
  if (tid == 0) mbar_init(&mbar, 1);
  if (warp == 0) {
    tmem_alloc(&tbase_s, NCOLS);
    tmem_relinquish();
  }
  float mu[N_IN], isg[N_IN];
#pragma unroll
  for (int k = 0; k < N_IN; ++k) {
    mu[k] = theta[OFF_MU + k];
    isg[k] = theta[OFF_ISG + k];
  }
  const float b4_0 = theta[OFF_B4], b4_1 = theta[OFF_B4 + 1];
  publish_tiles();
  const uint32_t tb = tbase_s;
  uint32_t phase = 0;
  float loss_acc = 0.0f, db4_0 = 0.0f, db4_1 = 0.0f;
  bool ok = true;
  const int ntiles = (n + TROWS - 1) / TROWS;
  const uint32_t ID64 = idesc_bf16(128, 64), ID16 = idesc_bf16(128, 16), ID80 = idesc_bf16(128, 80);

  int it = 0;
  for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it) {
    const int row = tile * TROWS + tid;
    const bool valid = row < n;
    float xh[N_IN];
#pragma unroll
    for (int k = 0; k < N_IN; ++k) xh[k] = valid ? (X[(size_t)row * N_IN + k] - mu[k]) * isg[k] : 0.0f;
    *reinterpret_cast<uint4*>(sm + S_A0 + tile_off(tid, 0, 16)) =
        make_uint4(pack_bf16x2(xh[0], xh[1]), pack_bf16x2(xh[2], xh[3]), pack_bf16x2(xh[4], 0.0f), 0u);
    *reinterpret_cast<uint4*>(sm + S_A0 + tile_off(tid, 8, 16)) = make_uint4(0u, 0u, 0u, 0u);
    if (TRAIN) {
#pragma unroll
      for (int k = 0; k < N_IN; ++k) st_bf16(sm, S_X0T + tile_off(k, tid, 128), xh[k]);
    }
    publish_tiles();

    // ---- forward ----
    if (tid == 0) {
      mma_bf16(tb + C_Z1, kdesc(s0 + S_A0, 16, 0), kdesc(s0 + S_W1, 16, 0), ID64, 0u);
      mma_commit(&mbar);
    }
    if (!(ok = wait_mma(&mbar, phase))) break;
    hidden_epilogue(tb, C_Z1, bias_s[0], sm, S_X1T, TRAIN);
    publish_tiles();
    if (tid == 0) {
      for (uint32_t s = 0; s < 4; ++s)
        mma_bf16(tb + C_Z2, kdesc(s0 + S_AH, 64, s), kdesc(s0 + S_W2, 64, s), ID64, s > 0);
      mma_commit(&mbar);
    }
    if (!(ok = wait_mma(&mbar, phase))) break;
    hidden_epilogue(tb, C_Z2, bias_s[1], sm, S_X2T, TRAIN);
    publish_tiles();
    if (tid == 0) {
      for (uint32_t s = 0; s < 4; ++s)
        mma_bf16(tb + C_Z3, kdesc(s0 + S_AH, 64, s), kdesc(s0 + S_W3, 64, s), ID64, s > 0);
      mma_commit(&mbar);
    }
    if (!(ok = wait_mma(&mbar, phase))) break;
    hidden_epilogue(tb, C_Z3, bias_s[2], sm, S_X3T, TRAIN);
    publish_tiles();
    if (tid == 0) {
      for (uint32_t s = 0; s < 4; ++s)
        mma_bf16(tb + C_O, kdesc(s0 + S_AH, 64, s), kdesc(s0 + S_W4, 64, s), ID16, s > 0);
      mma_commit(&mbar);
    }
    if (!(ok = wait_mma(&mbar, phase))) break;
    float o[16];
    tmem_ld16(taddr(tb, 32u * warp, C_O), o);
    const float o0 = o[0] + b4_0, o1 = o[1] + b4_1;
    if (!TRAIN) {
      if (valid) {
        out[(size_t)row * 2] = o0;
        out[(size_t)row * 2 + 1] = o1;
      }
      // the next tile rewrites A0 and the output columns only after every
      // thread has read them
      fence_before_sync();
      __syncthreads();
      fence_after_sync();
      continue;
    }

    // ---- backward ----
    float r0 = 0.0f, r1 = 0.0f;
    if (valid) {
      const float e0 = o0 - Y[(size_t)row * 2], e1 = o1 - Y[(size_t)row * 2 + 1];
      r0 = e0 * Mk[(size_t)row * 2];
      r1 = e1 * Mk[(size_t)row * 2 + 1];
      loss_acc += r0 * e0 + r1 * e1;
    }
    const float dz0 = r0 * inv_n, dz1 = r1 * inv_n;
    db4_0 += dz0;
    db4_1 += dz1;
    *reinterpret_cast<uint4*>(sm + S_DZ + tile_off(tid, 0, 16)) = make_uint4(pack_bf16x2(dz0, dz1), 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(sm + S_DZ + tile_off(tid, 8, 16)) = make_uint4(0u, 0u, 0u, 0u);
    st_bf16(sm, S_DZT + tile_off(64, tid, 128), dz0);
    st_bf16(sm, S_DZT + tile_off(65, tid, 128), dz1);
    publish_tiles();
    if (tid == 0) {
      // dW4 (rows 64-65 of the product; rows 0-63 are discarded)
      for (uint32_t s = 0; s < 8; ++s)
        mma_bf16(tb + C_DW4, kdesc(s0 + S_DZT, 128, s), kdesc(s0 + S_X3T, 128, s), ID64, (it > 0 || s > 0));
      // dA3 = dZ4 W4
      mma_bf16(tb + C_DA, kdesc(s0 + S_DZ, 16, 0), kdesc(s0 + S_W4T, 16, 0), ID64, 0u);
      mma_commit(&mbar);
    }
    if (!(ok = wait_mma(&mbar, phase))) break;
    backward_epilogue(tb, C_Z3, bias_s[2], sm, true);
    publish_tiles();
    if (tid == 0) {
      for (uint32_t s = 0; s < 8; ++s)
        mma_bf16(tb + C_DW3, kdesc(s0 + S_DZT, 128, s), kdesc(s0 + S_X2T, 128, s), ID80, (it > 0 || s > 0));
      for (uint32_t s = 0; s < 4; ++s)
        mma_bf16(tb + C_DA, kdesc(s0 + S_DZ, 64, s), kdesc(s0 + S_W3T, 64, s), ID64, s > 0);
      mma_commit(&mbar);
    }
    if (!(ok = wait_mma(&mbar, phase))) break;
    backward_epilogue(tb, C_Z2, bias_s[1], sm, true);
    publish_tiles();
    if (tid == 0) {
      for (uint32_t s = 0; s < 8; ++s)
        mma_bf16(tb + C_DW2, kdesc(s0 + S_DZT, 128, s), kdesc(s0 + S_X1T, 128, s), ID80, (it > 0 || s > 0));
      for (uint32_t s = 0; s < 4; ++s)
        mma_bf16(tb + C_DA, kdesc(s0 + S_DZ, 64, s), kdesc(s0 + S_W2T, 64, s), ID64, s > 0);
      mma_commit(&mbar);
    }
    if (!(ok = wait_mma(&mbar, phase))) break;
    backward_epilogue(tb, C_Z1, bias_s[0], sm, false);
    publish_tiles();
    if (tid == 0) {
      for (uint32_t s = 0; s < 8; ++s)
        mma_bf16(tb + C_DW1, kdesc(s0 + S_DZT, 128, s), kdesc(s0 + S_X0T, 128, s), ID16, (it > 0 || s > 0));
      mma_commit(&mbar);
    }
    if (!(ok = wait_mma(&mbar, phase))) break;
  }

  if (TRAIN && ok) {
    float* P = part + (size_t)blockIdx.x * N_PARAMS;
    if (it == 0) {  // no tile: zero gradient
      for (int p = tid; p < N_PARAMS; p += TROWS) P[p] = 0.0f;
    } else {
      if (tid < 2 * N_IN) P[tid] = 0.0f;
      if (warp < 2) {  // rows 0-63: hidden units of layers 1-3
        const int i = tid;
        float v[16];
        tmem_ld16(taddr(tb, 32u * warp, C_DW1), v);
#pragma unroll
        for (int j = 0; j < N_IN; ++j) P[OFF_W1 + i * N_IN + j] = v[j];
        P[OFF_B1 + i] = v[N_IN];
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          tmem_ld16(taddr(tb, 32u * warp, C_DW2 + 16u * c), v);
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int col = 16 * c + j;
            if (col < N_H) P[OFF_W2 + i * N_H + col] = v[j];
            else if (col == N_H) P[OFF_B2 + i] = v[j];
          }
          tmem_ld16(taddr(tb, 32u * warp, C_DW3 + 16u * c), v);
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int col = 16 * c + j;
            if (col < N_H) P[OFF_W3 + i * N_H + col] = v[j];
            else if (col == N_H) P[OFF_B3 + i] = v[j];
          }
        }
      } else if (warp == 2) {  // rows 64-65: output units of layer 4
        const int k = tid - 64;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float v[16];
          tmem_ld16(taddr(tb, 64u, C_DW4 + 16u * c), v);
          if (k < N_OUT) {
#pragma unroll
            for (int j = 0; j < 16; ++j) P[OFF_W4 + k * N_H + 16 * c + j] = v[j];
          }
        }
      }
      // output bias gradient and loss: fixed-order block reduction
#pragma unroll
      for (int o2 = 16; o2 > 0; o2 >>= 1) {
        db4_0 += __shfl_xor_sync(0xffffffffu, db4_0, o2);
        db4_1 += __shfl_xor_sync(0xffffffffu, db4_1, o2);
        loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, o2);
      }
      if (lane == 0) {
        red_s[warp][0] = db4_0;
        red_s[warp][1] = db4_1;
        red_s[warp][2] = loss_acc;
      }
      __syncthreads();
      if (tid == 0) {
        float a = 0.0f, b = 0.0f, l = 0.0f;
        for (int w = 0; w < 4; ++w) {
          a += red_s[w][0];
          b += red_s[w][1];
          l += red_s[w][2];
        }
        P[OFF_B4] = a;
        P[OFF_B4 + 1] = b;
        part[(size_t)MAX_GRID * N_PARAMS + blockIdx.x] = 0.5f * l * inv_n;
      }
    }
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0) tmem_dealloc(tb, NCOLS);
}

__global__ void k_mlp_adam(const float* __restrict__ part, int nblk, float* __restrict__ theta,
                           float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2, float eps,
                           float c1, float c2, float* __restrict__ grad_out, float* __restrict__ loss_out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < N_PARAMS) {
    float g = 0.0f;
    for (int c = 0; c < nblk; ++c) g += part[(size_t)c * N_PARAMS + p];
    if (grad_out) grad_out[p] = g;
    if (m && p >= 2 * N_IN) {
      const float mm = b1 * m[p] + (1.0f - b1) * g;
      const float vv = b2 * v[p] + (1.0f - b2) * g * g;
      m[p] = mm;
      v[p] = vv;
      theta[p] -= lr * (mm * c1) / (sqrtf(vv * c2) + eps);
    }
  }
  if (p == 0 && loss_out) {
    float l = 0.0f;
    for (int c = 0; c < nblk; ++c) l += part[(size_t)MAX_GRID * N_PARAMS + c];
    *loss_out = l;
  }
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

int launch(bool train, const float* theta, const float* X, const float* Y, const float* M, int64_t n, float* out,
           float* ws, cudaStream_t st, int* grid_out) {
  const int ntiles = (int)((n + TROWS - 1) / TROWS);
  int sms = sm_count();
  if (sms <= 0) return CGDEM_E_CUDA;
  const int grid = ntiles < sms ? ntiles : (sms < MAX_GRID ? sms : MAX_GRID);
  *grid_out = grid;
  if (grid == 0) return CGDEM_OK;
  int* err = reinterpret_cast<int*>(ws + (size_t)MAX_GRID * (N_PARAMS + 1));
  const size_t smem = (train ? S_END : S_INF_END) + 1024;
  cudaError_t e;
  if (train) {
    e = cudaFuncSetAttribute(k_mlp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      k_mlp<true><<<grid, TROWS, smem, st>>>(theta, X, Y, M, (int)n, 1.0f / (float)n, nullptr, ws, err);
  } else {
    e = cudaFuncSetAttribute(k_mlp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      k_mlp<false><<<grid, TROWS, smem, st>>>(theta, X, nullptr, nullptr, (int)n, 0.0f, out, ws, err);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "cgdem_mlp: launch failed: %s\n", cudaGetErrorString(e));
    return CGDEM_E_CUDA;
  }
  return CGDEM_OK;
}

constexpr int64_t MLP_MAX_N = (int64_t)1 << 28;

}  // namespace

namespace cgdem {

struct ClosureRange {
  float lo[5], hi[5], cd_max, cg_max;
};

// The network blob of the fused force kernel: the weight tiles exactly as the
// kernel's shared memory holds them, then biases, standardisation, input
// range and correction bounds in FP32.
__global__ void k_closure_pack(const float* __restrict__ th, ClosureRange r, uint8_t* __restrict__ blob) {
  using namespace closure;
  for (int e = threadIdx.x; e < 64 * 16; e += blockDim.x) {
    const int i = e >> 4, j = e & 15;
    st_bf16(blob, tile_off(i, j, 16), j < N_IN ? th[OFF_W1 + i * N_IN + j] : 0.0f);
  }
  for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
    const int i = e >> 6, j = e & 63;
    st_bf16(blob, 2048 + tile_off(i, j, 64), th[OFF_W2 + e]);
    st_bf16(blob, 10240 + tile_off(i, j, 64), th[OFF_W3 + e]);
  }
  for (int e = threadIdx.x; e < 16 * 64; e += blockDim.x) {
    const int k = e >> 6, j = e & 63;
    st_bf16(blob, 18432 + tile_off(k, j, 64), k < N_OUT ? th[OFF_W4 + k * N_H + j] : 0.0f);
  }
  float* P = reinterpret_cast<float*>(blob + CL_TILES);
  for (int e = threadIdx.x; e < 232; e += blockDim.x) {
    float v = 0.0f;
    if (e < 64) v = th[OFF_B1 + e];
    else if (e < 128) v = th[OFF_B2 + e - 64];
    else if (e < 192) v = th[OFF_B3 + e - 128];
    else if (e < (int)CL_P_B4 + 2) v = th[OFF_B4 + e - (int)CL_P_B4];
    else if (e >= (int)CL_P_MU && e < (int)CL_P_MU + 5) v = th[OFF_MU + e - (int)CL_P_MU];
    else if (e >= (int)CL_P_ISG && e < (int)CL_P_ISG + 5) v = th[OFF_ISG + e - (int)CL_P_ISG];
    else if (e >= (int)CL_P_LO && e < (int)CL_P_LO + 5) v = r.lo[e - (int)CL_P_LO];
    else if (e >= (int)CL_P_HI && e < (int)CL_P_HI + 5) v = r.hi[e - (int)CL_P_HI];
    else if (e == (int)CL_P_CMAX) v = r.cd_max;
    else if (e == (int)CL_P_CMAX + 1) v = r.cg_max;
    P[e] = v;
  }
}

void launch_closure_pack(const float* theta, const float* lo, const float* hi, float cd_max, float cg_max,
                         uint8_t* blob, cudaStream_t s) {
  ClosureRange r;
  for (int k = 0; k < 5; ++k) {
    r.lo[k] = lo[k];
    r.hi[k] = hi[k];
  }
  r.cd_max = cd_max;
  r.cg_max = cg_max;
  k_closure_pack<<<1, 256, 0, s>>>(theta, r, blob);
}

}  // namespace cgdem

extern "C" int cgdem_mlp_workspace_size(size_t* bytes) {
  if (!bytes) return CGDEM_E_INVALID;
  *bytes = ((size_t)MAX_GRID * (N_PARAMS + 1) + 64) * sizeof(float);
  return CGDEM_OK;
}

extern "C" int cgdem_mlp_forward(const float* theta, const float* X, int64_t n, float* out, void* workspace,
                                 size_t workspace_bytes, void* stream) {
  size_t need = 0;
  cgdem_mlp_workspace_size(&need);
  if (!theta || (n > 0 && (!X || !out)) || n < 0 || n > MLP_MAX_N || !workspace || workspace_bytes < need)
    return CGDEM_E_INVALID;
  int grid = 0;
  return launch(false, theta, X, nullptr, nullptr, n, out, static_cast<float*>(workspace),
                reinterpret_cast<cudaStream_t>(stream), &grid);
}

extern "C" int cgdem_mlp_train_step(float* theta, float* adam_m, float* adam_v, int64_t t, double lr,
                                    const float* X, const float* Y, const float* M, int64_t n, float* grad_out,
                                    float* loss_out, void* workspace, size_t workspace_bytes, void* stream) {
  size_t need = 0;
  cgdem_mlp_workspace_size(&need);
  if (!theta || !X || !Y || !M || n <= 0 || n > MLP_MAX_N || !workspace || workspace_bytes < need ||
      ((adam_m == nullptr) != (adam_v == nullptr)) || (adam_m && (t < 1 || !(lr >= 0.0))))
    return CGDEM_E_INVALID;
  float* ws = static_cast<float*>(workspace);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int grid = 0;
  int r = launch(true, theta, X, Y, M, n, nullptr, ws, st, &grid);
  if (r != CGDEM_OK) return r;
  const double b1 = 0.9, b2 = 0.999;
  const double c1 = adam_m ? 1.0 / (1.0 - pow(b1, (double)t)) : 0.0;
  const double c2 = adam_m ? 1.0 / (1.0 - pow(b2, (double)t)) : 0.0;
  k_mlp_adam<<<(N_PARAMS + 255) / 256, 256, 0, st>>>(ws, grid, theta, adam_m, adam_v, (float)lr, (float)b1,
                                                      (float)b2, 1e-8f, (float)c1, (float)c2, grad_out, loss_out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "cgdem_mlp_train_step: launch failed: %s\n", cudaGetErrorString(e));
    return CGDEM_E_CUDA;
  }
  return CGDEM_OK;
}

extern "C" int cgdem_mlp_status(void* workspace, void* stream) {
  if (!workspace) return CGDEM_E_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int* err = reinterpret_cast<int*>(static_cast<float*>(workspace) + (size_t)MAX_GRID * (N_PARAMS + 1));
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return CGDEM_E_CUDA;
  if (h) {
    cudaMemsetAsync(err, 0, sizeof(int), st);
    cudaStreamSynchronize(st);
    return CGDEM_E_TIMEOUT;
  }
  return CGDEM_OK;
}
