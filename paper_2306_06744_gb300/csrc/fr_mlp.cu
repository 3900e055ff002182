// fr_mlp.cu -- learned adaptation indicator: a per-element MLP that predicts the density-gradient
// indicator a few steps ahead (refine / keep / coarsen), so adaptation can run less often.
//
// Network: x (IN inputs) -> 64 -> 64 -> 64 -> 3 logits, GELU after the three hidden layers.
// Inputs, weights and activations are stored in BF16; every dot product accumulates in FP32.
// Parameters are one FP32 array (the optimiser's master copy), laid out
//   [W1 (64 x IN) | b1 (64) | W2 (64 x 64) | b2 | W3 (64 x 64) | b3 | W4 (3 x 64) | b4 (3)].
// Features of an element: density and pressure at the 3^dim Gauss-Legendre points of order 3
// (interpolated from the element's polynomial, so the same network serves every degree), as
// relative deviations from their means scaled by 100 (a 1% variation is 1.0), then the depth as
// (D - Dbase) / max(1, Dmax - Dbase): IN = 2*3^dim + 1 inputs (19 in 2D, 55 in 3D).
//
// Inference runs on the tensor cores (tcgen05, BF16 operands in shared memory, FP32 accumulators
// in tensor memory): batched over elements the layers are dense [128 x 64] x [64 x 64]
// contractions.  Training (per-sample forward/backward and the weight-gradient reduction) runs on
// the CUDA cores with FP32 FMA on BF16-rounded operands.
#include <cuda_bf16.h>

#include <cmath>

#include "fr_arith.cuh"
#include "fr_internal.cuh"
#include "fr_mlp.cuh"
#include "fr_tc.cuh"

namespace frg {

namespace {

constexpr int H = MLP_HIDDEN;
constexpr int NOUT = 3;
constexpr int MLP_T = 128;  // threads (samples) per block

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// GELU with the exact erf form and its derivative
__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

struct Lay {
  int in;
  int oW1, ob1, oW2, ob2, oW3, ob3, oW4, ob4, total;
};
__host__ __device__ inline Lay lay(int in) {
  Lay L;
  L.in = in;
  L.oW1 = 0;
  L.ob1 = L.oW1 + H * in;
  L.oW2 = L.ob1 + H;
  L.ob2 = L.oW2 + H * H;
  L.oW3 = L.ob2 + H;
  L.ob3 = L.oW3 + H * H;
  L.oW4 = L.ob3 + H;
  L.ob4 = L.oW4 + NOUT * H;
  L.total = L.ob4 + NOUT;
  return L;
}

// features from the FP64 state: the conserved variables are interpolated from the element's own
// points to the 3 Gauss-Legendre points per axis (I3 = 3 x n Lagrange matrix, as double-word
// constants), where density and pressure are taken
struct I3Mat {
  ff m[3][NPMAX];
};

// One thread per element, in double-word arithmetic (pairs of floats, ~48-bit significand, on
// the FP32 pipes; the state converts from FP64 by integer operations): the features are relative
// deviations of nearly equal values, which FP32 alone would swamp with rounding noise, while FP64
// on GB300 runs at 1/58 of the FP32 rate.  The interpolation to the 3^dim sample points is
// sum-factorised (one axis at a time: n^dim -> 3 n^(dim-1) -> ... -> 3^dim values per variable);
// density is kept per sample point, the squared momentum accumulated, and pressure formed when
// the energy arrives.  In 3D the first two axes are done per z-slice, so only 3^2 n values stay
// live.
template <int DIM, int NP>
__global__ void __launch_bounds__(128) k_features(const double* __restrict__ u, const uint64_t* __restrict__ keys,
                                                  int64_t M, KG g, int Dbase, double gamma,
                                                  const __grid_constant__ I3Mat I3, __nv_bfloat16* __restrict__ X) {
  constexpr int N = DIM == 2 ? NP * NP : NP * NP * NP;
  constexpr int NZ = DIM == 2 ? 1 : NP;  // z-slices
  constexpr int S = DIM == 2 ? 9 : 27;   // sample points, t = s0 + 3 s1 (+ 9 s2)
  constexpr int NV = DIM + 2, IN = 2 * S + 1;
  int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= M) return;
  const double* q = u + e * NV * N;
  const ff gm1 = ff_from_double(gamma - 1.0), half = {0.5f, 0.f}, zero = {0.f, 0.f};
  ff rho[S], ke[S];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    // b[i2][s1][s0] = sum_i1 I[s1][i1] sum_i0 I[s0][i0] q[i2][i1][i0]
    ff b[NZ][3][3];
#pragma unroll
    for (int i2 = 0; i2 < NZ; ++i2) {
      ff a[NP][3];
#pragma unroll
      for (int i1 = 0; i1 < NP; ++i1) {
        ff x[NP];
#pragma unroll
        for (int i0 = 0; i0 < NP; ++i0) x[i0] = ff_from_double(q[v * N + (i2 * NP + i1) * NP + i0]);
#pragma unroll
        for (int s0 = 0; s0 < 3; ++s0) {
          ff acc = zero;
#pragma unroll
          for (int i0 = 0; i0 < NP; ++i0) acc = fma_t(I3.m[s0][i0], x[i0], acc);
          a[i1][s0] = acc;
        }
      }
#pragma unroll
      for (int s1 = 0; s1 < 3; ++s1)
#pragma unroll
        for (int s0 = 0; s0 < 3; ++s0) {
          ff acc = zero;
#pragma unroll
          for (int i1 = 0; i1 < NP; ++i1) acc = fma_t(I3.m[s1][i1], a[i1][s0], acc);
          b[i2][s1][s0] = acc;
        }
    }
#pragma unroll
    for (int t = 0; t < S; ++t) {
      const int s0 = t % 3, s1 = (t / 3) % 3, s2 = t / 9;
      ff c;
      if (DIM == 2) {
        c = b[0][s1][s0];
      } else {
        c = zero;
#pragma unroll
        for (int i2 = 0; i2 < NZ; ++i2) c = fma_t(I3.m[s2][i2], b[i2][s1][s0], c);
      }
      if (v == 0) {
        rho[t] = c;
        ke[t] = zero;
      } else if (v < NV - 1) {
        ke[t] = fma_t(c, c, ke[t]);
      } else {
        ke[t] = gm1 * (c - half * ke[t] / rho[t]);  // pressure
      }
    }
  }
  ff rm = zero, pm = zero;
#pragma unroll
  for (int t = 0; t < S; ++t) {
    rm = rm + rho[t];
    pm = pm + ke[t];
  }
  // 100 (q_t - mean) / mean = (q_t - mean) * (100 S / sum)
  const ff hs = ff_from_double(100.0 * S);
  const ff fr_ = hs / rm, fp_ = hs / pm;
  const ff inv_s = ff_from_double(1.0 / S);
  rm = rm * inv_s;
  pm = pm * inv_s;
  __nv_bfloat16* x = X + e * IN;
#pragma unroll
  for (int t = 0; t < S; ++t) {
    const ff dr = (rho[t] - rm) * fr_, dp = (ke[t] - pm) * fp_;
    x[t] = __float2bfloat16_rn(dr.h + dr.l);
    x[S + t] = __float2bfloat16_rn(dp.h + dp.l);
  }
  int span = g.Dmax - Dbase > 0 ? g.Dmax - Dbase : 1;
  x[2 * S] = __float2bfloat16_rn(float(g.depth(keys[e]) - Dbase) / float(span));
}

// shared-memory copy of the BF16-rounded weights as floats
__device__ void load_weights(const float* __restrict__ P, int total, float* sw) {
  for (int k = threadIdx.x; k < total; k += blockDim.x) sw[k] = bf16r(P[k]);
}

// first layer: z[i] = b[i] + sum_k W[i][k] x_k, x read from the BF16 input row
__device__ __forceinline__ void layer_in(const float* W, const float* b, const __nv_bfloat16* x,
                                         int in, float (&z)[H]) {
#pragma unroll
  for (int i = 0; i < H; ++i) z[i] = b[i];
  for (int k = 0; k < in; ++k) {
    float xk = __bfloat162float(x[k]);
#pragma unroll
    for (int i = 0; i < H; ++i) z[i] = fmaf(W[i * in + k], xk, z[i]);
  }
}
// hidden layer: z[i] = b[i] + sum_k W[i][k] a_k
__device__ __forceinline__ void layer_h(const float* W, const float* b, const float (&a)[H],
                                        float (&z)[H]) {
#pragma unroll
  for (int i = 0; i < H; ++i) z[i] = b[i];
#pragma unroll
  for (int k = 0; k < H; ++k) {
#pragma unroll
    for (int i = 0; i < H; ++i) z[i] = fmaf(W[i * H + k], a[k], z[i]);
  }
}
__device__ __forceinline__ void act(const float (&z)[H], float (&a)[H]) {
#pragma unroll
  for (int i = 0; i < H; ++i) a[i] = bf16r(gelu(z[i]));
}
__device__ __forceinline__ void layer_out(const float* W, const float* b, const float (&a)[H],
                                          float (&z)[NOUT]) {
#pragma unroll
  for (int c = 0; c < NOUT; ++c) {
    float t = b[c];
#pragma unroll
    for (int k = 0; k < H; ++k) t = fmaf(W[c * H + k], a[k], t);
    z[c] = t;
  }
}

// Tensor-core forward.  Each block keeps the four weight matrices in shared memory as BF16 in the
// K-major core-matrix layout of fr_tc.cuh (W1 zero-padded to 64 inputs, W4 to 16 outputs) and
// loops over tiles of 128 samples.  The tile's feature rows are one contiguous block, fetched by a
// bulk copy into one of two staging buffers while the previous tile is computed.  Per tile the
// rows are rewritten into the activation tile A; per layer one thread issues the K/16 MMAs of
// A * W^T into a 128 x 64 FP32 accumulator in tensor memory and commits them to an mbarrier; once
// it completes, thread r reads row r of the accumulator (TMEM lane r), adds the bias, applies
// GELU, rounds to BF16 and writes the row back into A as the next layer's operand.  The output
// layer (N = 16, 3 used) gives the logits and the argmax flag.  A wait that does not complete
// within about a second sets *status, waits once more (bounded) for the copies and MMAs in
// flight, frees the tensor memory and ends the block.
constexpr int TC_ROWS = 128, TC_TMEM_COLS = 64;
constexpr long long TC_WAIT_CYCLES = 2000000000ll;
constexpr int TC_W1 = 0, TC_W2 = 8192, TC_W3 = 16384, TC_W4 = 24576, TC_A = 26624, TC_X0 = 43008;
// shared-memory plan for `in` inputs: two staging buffers of 128*in BF16 (1024-byte granules),
// then the biases, the three mbarriers and the TMEM address; plus 1024 bytes of alignment slack
struct TcPlan {
  int x1, bias, mbar, bytes;
};
__host__ __device__ inline TcPlan tc_plan(int in) {
  const int xb = (TC_ROWS * in * 2 + 1023) / 1024 * 1024;
  TcPlan q;
  q.x1 = TC_X0 + xb;
  q.bias = q.x1 + xb;
  q.mbar = q.bias + 208 * 4;
  q.bytes = q.mbar + 32 + 1024;
  return q;
}

__global__ void __launch_bounds__(TC_ROWS) k_mlp_forward_tc(const float* __restrict__ P, int in,
                                                            const __nv_bfloat16* __restrict__ X, int64_t n,
                                                            float* __restrict__ logits,
                                                            int8_t* __restrict__ flags, int* __restrict__ status) {
  extern __shared__ unsigned char sm_raw[];
  // 1024-byte aligned base for the operand tiles
  unsigned char* sm = sm_raw + ((1024 - (tc::smem_addr(sm_raw) & 1023)) & 1023);
  const int t = threadIdx.x, warp = t >> 5;
  const Lay L = lay(in);
  const TcPlan Q = tc_plan(in);
  const int64_t ntiles = (n + TC_ROWS - 1) / TC_ROWS;
  const uint32_t mb = tc::smem_addr(sm + Q.mbar);  // MMA completion
  const uint32_t fb[2] = {mb + 8, mb + 16};        // feature copies into the staging buffers
  const int xoff[2] = {TC_X0, Q.x1};
  // a tile is fetched by a bulk copy when it is full (its 256*in bytes start 16-byte aligned when
  // X does); the last, partial tile is read by the threads
  const bool bulk_ok = (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  auto tile_bulk = [&](int64_t tile) { return bulk_ok && (tile + 1) * TC_ROWS <= n; };
  auto fetch = [&](int64_t tile, int b) {
    tc::fence_proxy_async();
    tc::bulk_g2s(tc::smem_addr(sm + xoff[b]), X + tile * TC_ROWS * in, uint32_t(TC_ROWS * in * 2), fb[b]);
  };
  // copies in flight per staging buffer (the issue conditions are uniform over the block)
  bool pend[2] = {blockIdx.x < ntiles && tile_bulk(blockIdx.x), false};
  if (t == 0) {
    tc::mbar_init(mb, 1);
    tc::mbar_init(fb[0], 1);
    tc::mbar_init(fb[1], 1);
    if (pend[0]) fetch(blockIdx.x, 0);
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(sm + Q.mbar + 24), TC_TMEM_COLS);
  auto put = [&](int off, int r, int k, float v) {
    *reinterpret_cast<__nv_bfloat16*>(sm + off + tc::canon_off(r, k)) = __float2bfloat16_rn(v);
  };
  for (int idx = t; idx < H * 64; idx += TC_ROWS) {
    const int o = idx >> 6, k = idx & 63;
    put(TC_W1, o, k, k < in ? P[L.oW1 + o * in + k] : 0.f);
    put(TC_W2, o, k, P[L.oW2 + o * H + k]);
    put(TC_W3, o, k, P[L.oW3 + o * H + k]);
    if (o < 16) put(TC_W4, o, k, o < NOUT ? P[L.oW4 + o * H + k] : 0.f);
  }
  float* sb = reinterpret_cast<float*>(sm + Q.bias);  // b1 | b2 | b3 | b4 (16), BF16-rounded
  for (int i = t; i < H; i += TC_ROWS) {
    sb[i] = bf16r(P[L.ob1 + i]);
    sb[H + i] = bf16r(P[L.ob2 + i]);
    sb[2 * H + i] = bf16r(P[L.ob3 + i]);
  }
  if (t < 16) sb[3 * H + t] = t < NOUT ? bf16r(P[L.ob4 + t]) : 0.f;
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(sm + Q.mbar + 24);
  const uint32_t tlane = tmem + (uint32_t(warp * 32) << 16);  // this warp's 32 TMEM lanes
  const uint32_t sA = tc::smem_addr(sm + TC_A);
  const int K1 = in <= 32 ? 32 : 64;
  uint32_t phase = 0, fphase[2] = {0, 0};
  bool failed = false, mma_pend = false;
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x, ++it) {
    const int b = it & 1;
    const int64_t row0 = tile * TC_ROWS;
    const int nrow = int(n - row0 < TC_ROWS ? n - row0 : TC_ROWS);
    const unsigned char* xs;  // this tile's rows, contiguous BF16
    if (pend[b]) {
      const bool ok = tc::mbar_wait(fb[b], fphase[b], TC_WAIT_CYCLES);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      fphase[b] ^= 1;
      pend[b] = false;
      xs = sm + xoff[b];
    } else {
      xs = reinterpret_cast<const unsigned char*>(X + row0 * in);
    }
    // the next tile of this block goes into the other staging buffer, read in the last iteration
    if (tile + gridDim.x < ntiles && tile_bulk(tile + gridDim.x)) {
      pend[b ^ 1] = true;
      if (t == 0) fetch(tile + gridDim.x, b ^ 1);
    }
    // row t of the tile -> row t of A (zero rows past the end, zero columns past `in`)
    {
      const __nv_bfloat16* xr = reinterpret_cast<const __nv_bfloat16*>(xs) + t * in;
      for (int k0 = 0; k0 < K1; k0 += 8) {
        uint32_t pk[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int k = k0 + 2 * j;
          __nv_bfloat162 h2;
          h2.x = (t < nrow && k < in) ? xr[k] : __float2bfloat16_rn(0.f);
          h2.y = (t < nrow && k + 1 < in) ? xr[k + 1] : __float2bfloat16_rn(0.f);
          pk[j] = *reinterpret_cast<uint32_t*>(&h2);
        }
        *reinterpret_cast<uint4*>(sm + TC_A + tc::canon_off(t, k0)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      }
    }
    for (int layer = 0; layer < 4; ++layer) {
      tc::fence_proxy_async();
      tc::fence_before_sync();
      __syncthreads();
      if (t == 0) {
        tc::fence_after_sync();
        const int nk = layer == 0 ? K1 / 16 : H / 16;
        const uint32_t sW = tc::smem_addr(sm + (layer == 0 ? TC_W1 : layer == 1 ? TC_W2 : layer == 2 ? TC_W3 : TC_W4));
        const uint32_t id = tc::idesc_bf16(TC_ROWS, layer == 3 ? 16 : H);
        for (int ks = 0; ks < nk; ++ks)
          tc::mma_bf16(tmem, tc::sdesc(sA + ks * 2 * tc::LBO), tc::sdesc(sW + ks * 2 * tc::LBO), id, ks > 0);
        tc::commit(mb);
      }
      mma_pend = true;
      const bool ok = tc::mbar_wait(mb, phase, TC_WAIT_CYCLES);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      phase ^= 1;
      mma_pend = false;
      tc::fence_after_sync();
      if (layer < 3) {
        const float* bl = sb + H * layer;
        uint32_t r[4][16];
#pragma unroll
        for (int q = 0; q < 4; ++q) tc::tmem_ld16(tlane + uint32_t(16 * q), r[q]);
        tc::tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          uint32_t pk[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int c = 16 * q + 2 * j;
            __nv_bfloat162 h2 = __floats2bfloat162_rn(gelu(__uint_as_float(r[q][2 * j]) + bl[c]),
                                                      gelu(__uint_as_float(r[q][2 * j + 1]) + bl[c + 1]));
            pk[j] = *reinterpret_cast<uint32_t*>(&h2);
          }
          *reinterpret_cast<uint4*>(sm + TC_A + tc::canon_off(t, 16 * q)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
          *reinterpret_cast<uint4*>(sm + TC_A + tc::canon_off(t, 16 * q + 8)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
      } else {
        uint32_t r[16];
        tc::tmem_ld16(tlane, r);
        tc::tmem_wait_ld();
        if (t < nrow) {
          const int64_t row = row0 + t;
          float o[NOUT];
#pragma unroll
          for (int c = 0; c < NOUT; ++c) o[c] = __uint_as_float(r[c]) + sb[3 * H + c];
          if (logits)
            for (int c = 0; c < NOUT; ++c) logits[row * NOUT + c] = o[c];
          if (flags) {
            int best = 0;
            for (int c = 1; c < NOUT; ++c)
              if (o[c] > o[best]) best = c;
            flags[row] = int8_t(best - 1);  // class 0 coarsen, 1 keep, 2 refine
          }
        }
      }
    }
  }
  if (failed) {
    if (t == 0) atomicExch(status, 1);
    // bounded waits for what may still be in flight (the block's shared memory must not be
    // released under a copy): the MMAs of the failed wait and the pending feature copies
    if (mma_pend) tc::mbar_wait(mb, phase, TC_WAIT_CYCLES);
    for (int q = 0; q < 2; ++q)
      if (pend[q]) tc::mbar_wait(fb[q], fphase[q], TC_WAIT_CYCLES);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_free(tmem, TC_TMEM_COLS);
  }
}

// training, per sample: forward, weighted softmax cross-entropy, backward to every layer's
// pre-activation gradient.  Stores the inputs of every layer (A0..A3), the pre-activations
// (Z1..Z3) and the gradients (D1..D4) for the weight-gradient reduction, and the sample's loss.
__global__ void __launch_bounds__(MLP_T) k_mlp_fwd_bwd(const float* __restrict__ P, int in,
                                                       const __nv_bfloat16* __restrict__ X,
                                                       const int8_t* __restrict__ y, int64_t B,
                                                       float cw0, float cw1, float cw2, float inv_wsum,
                                                       float* __restrict__ A, float* __restrict__ Z,
                                                       float* __restrict__ D, float* __restrict__ loss) {
  extern __shared__ float sw[];
  const Lay L = lay(in);
  load_weights(P, L.total, sw);
  __syncthreads();
  int64_t b = int64_t(blockIdx.x) * MLP_T + threadIdx.x;
  if (b >= B) return;
  const int64_t HA = B * H;
  float* A0 = A;  // B x in, then A1..A3 (B x 64 each)
  float* A1 = A + B * in;
  float* A2 = A1 + HA;
  float* A3 = A2 + HA;
  float* Z1 = Z;
  float* Z2 = Z + HA;
  float* Z3 = Z2 + HA;
  float* D1 = D;  // B x 64 each, then D4: B x 3
  float* D2 = D1 + HA;
  float* D3 = D2 + HA;
  float* D4 = D3 + HA;
  const __nv_bfloat16* x = X + b * in;
  for (int k = 0; k < in; ++k) A0[b * in + k] = __bfloat162float(x[k]);
  float z[H], a[H], o[NOUT];
  layer_in(sw + L.oW1, sw + L.ob1, x, in, z);
  act(z, a);
#pragma unroll
  for (int i = 0; i < H; ++i) {
    Z1[b * H + i] = z[i];
    A1[b * H + i] = a[i];
  }
  layer_h(sw + L.oW2, sw + L.ob2, a, z);
  act(z, a);
#pragma unroll
  for (int i = 0; i < H; ++i) {
    Z2[b * H + i] = z[i];
    A2[b * H + i] = a[i];
  }
  layer_h(sw + L.oW3, sw + L.ob3, a, z);
  act(z, a);
#pragma unroll
  for (int i = 0; i < H; ++i) {
    Z3[b * H + i] = z[i];
    A3[b * H + i] = a[i];
  }
  layer_out(sw + L.oW4, sw + L.ob4, a, o);
  // softmax cross-entropy with class weights, normalised by the batch's total weight
  int cls = int(y[b]) + 1;
  float w = cls == 0 ? cw0 : (cls == 1 ? cw1 : cw2);
  float mx = fmaxf(o[0], fmaxf(o[1], o[2]));
  float e0 = expf(o[0] - mx), e1 = expf(o[1] - mx), e2 = expf(o[2] - mx);
  float sum = e0 + e1 + e2;
  float pz[NOUT] = {e0 / sum, e1 / sum, e2 / sum};
  loss[b] = -w * inv_wsum * logf(pz[cls]);
  float d4[NOUT];
#pragma unroll
  for (int c = 0; c < NOUT; ++c) {
    d4[c] = w * inv_wsum * (pz[c] - (c == cls ? 1.f : 0.f));
    D4[b * NOUT + c] = d4[c];
  }
  // backward: d3 = (W4^T d4) * gelu'(z3), d2 = (W3^T d3) * gelu'(z2), d1 = (W2^T d2) * gelu'(z1)
  float d[H], g[H];
#pragma unroll
  for (int k = 0; k < H; ++k) {
    float t = 0.f;
#pragma unroll
    for (int c = 0; c < NOUT; ++c) t = fmaf(sw[L.oW4 + c * H + k], d4[c], t);
    d[k] = t * gelu_d(Z3[b * H + k]);
    D3[b * H + k] = d[k];
  }
#pragma unroll
  for (int k = 0; k < H; ++k) g[k] = 0.f;
#pragma unroll
  for (int i = 0; i < H; ++i) {
#pragma unroll
    for (int k = 0; k < H; ++k) g[k] = fmaf(sw[L.oW3 + i * H + k], d[i], g[k]);
  }
#pragma unroll
  for (int k = 0; k < H; ++k) {
    d[k] = g[k] * gelu_d(Z2[b * H + k]);
    D2[b * H + k] = d[k];
    g[k] = 0.f;
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
#pragma unroll
    for (int k = 0; k < H; ++k) g[k] = fmaf(sw[L.oW2 + i * H + k], d[i], g[k]);
  }
#pragma unroll
  for (int k = 0; k < H; ++k) D1[b * H + k] = g[k] * gelu_d(Z1[b * H + k]);
}

// weight gradients, one thread per parameter, summing the batch in index order (deterministic)
__global__ void k_mlp_wgrad(int in, int64_t B, const float* __restrict__ A, const float* __restrict__ D,
                            float* __restrict__ G) {
  const Lay L = lay(in);
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= L.total) return;
  const int64_t HA = B * H;
  const float* A0 = A;
  const float* A1 = A + B * in;
  const float* A2 = A1 + HA;
  const float* A3 = A2 + HA;
  const float* D1 = D;
  const float* D2 = D1 + HA;
  const float* D3 = D2 + HA;
  const float* D4 = D3 + HA;
  const float *Ad = nullptr, *Dd = nullptr;
  int nin = 0, nout = H, i = 0, k = -1;
  if (t < L.ob1) { Ad = A0; Dd = D1; nin = in; i = (t - L.oW1) / in; k = (t - L.oW1) % in; }
  else if (t < L.oW2) { Dd = D1; i = t - L.ob1; }
  else if (t < L.ob2) { Ad = A1; Dd = D2; nin = H; i = (t - L.oW2) / H; k = (t - L.oW2) % H; }
  else if (t < L.oW3) { Dd = D2; i = t - L.ob2; }
  else if (t < L.ob3) { Ad = A2; Dd = D3; nin = H; i = (t - L.oW3) / H; k = (t - L.oW3) % H; }
  else if (t < L.oW4) { Dd = D3; i = t - L.ob3; }
  else if (t < L.ob4) { Ad = A3; Dd = D4; nin = H; nout = NOUT; i = (t - L.oW4) / H; k = (t - L.oW4) % H; }
  else { Dd = D4; nout = NOUT; i = t - L.ob4; }
  float s = 0.f;
  if (k >= 0) {
    for (int64_t b = 0; b < B; ++b) s = fmaf(Dd[b * nout + i], Ad[b * nin + k], s);
  } else {
    for (int64_t b = 0; b < B; ++b) s += Dd[b * nout + i];
  }
  G[t] = s;
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2, p -= lr mhat / (sqrt(vhat) + eps)
__global__ void k_adam(float* __restrict__ P, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ G, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  float g = G[t];
  float mt = b1 * m[t] + (1.f - b1) * g;
  float vt = b2 * v[t] + (1.f - b2) * g * g;
  m[t] = mt;
  v[t] = vt;
  P[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
}

// deterministic sum of the per-sample losses (one block, fixed order)
__global__ void k_sum(const float* __restrict__ x, int64_t n, float* __restrict__ out) {
  __shared__ float s[256];
  float a = 0.f;
  for (int64_t i = threadIdx.x; i < n; i += 256) a += x[i];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (int(threadIdx.x) < st) s[threadIdx.x] += s[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

size_t fwd_smem(int in) { return sizeof(float) * size_t(lay(in).total); }

}  // namespace

int mlp_param_count(int in) { return lay(in).total; }

int mlp_forward(const float* d_params, int in, const void* d_X, int64_t n, float* d_logits,
                int8_t* d_flags, int* d_status, cudaStream_t s, Err* err) {
  if (in < 1 || in > 64) return set_error(err, FR_EINVAL, "the MLP takes 1..64 inputs");
  if (n <= 0) return 0;
  int dev = 0;
  FR_CUDA(err, cudaGetDevice(&dev));
  const int smem = tc_plan(in).bytes;
  static int sms = 0, smem_sm = 0, resv = 0, regs = 0;
  if (sms == 0) {
    FR_CUDA(err, cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    FR_CUDA(err, cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev));
    FR_CUDA(err, cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    cudaFuncAttributes fa{};
    FR_CUDA(err, cudaFuncGetAttributes(&fa, k_mlp_forward_tc));
    regs = fa.numRegs > 0 ? fa.numRegs : 255;
    FR_CUDA(err, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  FR_CUDA(err, cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  // resident blocks per SM: shared memory, registers, and the SM's 512 tensor-memory columns of
  // which every block holds TC_TMEM_COLS
  int per = smem_sm / (smem + resv);
  const int by_regs = 65536 / (regs * TC_ROWS);
  if (per > by_regs) per = by_regs;
  if (per > 512 / TC_TMEM_COLS) per = 512 / TC_TMEM_COLS;
  const int64_t cap = int64_t(sms) * (per > 0 ? per : 1);
  const int64_t ntiles = (n + TC_ROWS - 1) / TC_ROWS;
  const unsigned grid = unsigned(ntiles < cap ? ntiles : cap);
  k_mlp_forward_tc<<<grid, TC_ROWS, smem, s>>>(d_params, in, static_cast<const __nv_bfloat16*>(d_X), n,
                                               d_logits, d_flags, d_status);
  FR_LAUNCH_CHECK(err);
  return 0;
}

int mlp_in_dim(int dim) { return 2 * (dim == 2 ? 9 : 27) + 1; }

int mlp_features(int dim, int p, const double* u, const uint64_t* keys, int64_t M, const KG& g,
                 int Dbase, double gamma, const DevOps& ops, void* d_X, cudaStream_t s, Err* err) {
  if (M <= 0) return 0;
  // Lagrange basis of the element's points evaluated at the 3-point Gauss-Legendre nodes
  I3Mat I3{};
  const double g3[3] = {-std::sqrt(0.6), 0.0, std::sqrt(0.6)};
  int np = p + 1;
  for (int t = 0; t < 3; ++t)
    for (int j = 0; j < np; ++j) {
      double pr = 1.0;
      for (int k = 0; k < np; ++k)
        if (k != j) pr *= (g3[t] - ops.x[k]) / (ops.x[j] - ops.x[k]);
      const float h = float(pr);  // double-word constant: hi + lo
      I3.m[t][j] = ff{h, float(pr - double(h))};
    }
  unsigned nb = unsigned((M + 127) / 128);
  __nv_bfloat16* X = static_cast<__nv_bfloat16*>(d_X);
#define FEAT(D_, N_) k_features<D_, N_><<<nb, 128, 0, s>>>(u, keys, M, g, Dbase, gamma, I3, X)
  if (dim == 2) {
    if (np == 2) FEAT(2, 2); else if (np == 3) FEAT(2, 3); else if (np == 4) FEAT(2, 4); else FEAT(2, 5);
  } else {
    if (np == 2) FEAT(3, 2); else if (np == 3) FEAT(3, 3); else if (np == 4) FEAT(3, 4); else FEAT(3, 5);
  }
#undef FEAT
  FR_LAUNCH_CHECK(err);
  return 0;
}

int mlp_train_step(float* d_params, float* d_m, float* d_v, int64_t step, int in, const void* d_X,
                   const int8_t* d_y, int64_t B, const float* cw, float lr, float* d_loss,
                   Alloc& A, cudaStream_t s, Err* err) {
  if (B <= 0) return set_error(err, FR_EINVAL, "empty batch");
  const Lay L = lay(in);
  Scratch S(&A);
  float* acts = S.get<float>(size_t(B) * (in + 3 * H));
  float* pre = S.get<float>(size_t(B) * 3 * H);
  float* dels = S.get<float>(size_t(B) * (3 * H + NOUT));
  float* G = S.get<float>(L.total);
  float* ls = S.get<float>(B);
  if (!acts || !pre || !dels || !G || !ls) return set_error(err, FR_ENOMEM, "training scratch");
  // class weights normalised by the batch's total weight: computed by the caller as cw[0..2]
  // and cw[3] = 1 / sum_b w_{y_b}
  size_t sm = fwd_smem(in);
  FR_CUDA(err, cudaFuncSetAttribute(k_mlp_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)));
  k_mlp_fwd_bwd<<<unsigned((B + MLP_T - 1) / MLP_T), MLP_T, sm, s>>>(
      d_params, in, static_cast<const __nv_bfloat16*>(d_X), d_y, B, cw[0], cw[1], cw[2], cw[3], acts,
      pre, dels, ls);
  FR_LAUNCH_CHECK(err);
  k_mlp_wgrad<<<unsigned((L.total + 127) / 128), 128, 0, s>>>(in, B, acts, dels, G);
  FR_LAUNCH_CHECK(err);
  const float b1 = 0.9f, b2 = 0.999f;
  float c1 = 1.f - std::pow(b1, float(step + 1)), c2 = 1.f - std::pow(b2, float(step + 1));
  k_adam<<<unsigned((L.total + 255) / 256), 256, 0, s>>>(d_params, d_m, d_v, G, L.total, lr, b1, b2,
                                                         1e-8f, c1, c2);
  FR_LAUNCH_CHECK(err);
  if (d_loss) {
    k_sum<<<1, 256, 0, s>>>(ls, B, d_loss);
    FR_LAUNCH_CHECK(err);
  }
  return 0;
}

int mlp_grad(const float* d_params, int in, const void* d_X, const int8_t* d_y, int64_t B,
             const float* cw, float* d_grad, float* d_loss, Alloc& A, cudaStream_t s, Err* err) {
  if (B <= 0) return set_error(err, FR_EINVAL, "empty batch");
  const Lay L = lay(in);
  Scratch S(&A);
  float* acts = S.get<float>(size_t(B) * (in + 3 * H));
  float* pre = S.get<float>(size_t(B) * 3 * H);
  float* dels = S.get<float>(size_t(B) * (3 * H + NOUT));
  float* ls = S.get<float>(B);
  if (!acts || !pre || !dels || !ls) return set_error(err, FR_ENOMEM, "gradient scratch");
  size_t sm = fwd_smem(in);
  FR_CUDA(err, cudaFuncSetAttribute(k_mlp_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)));
  k_mlp_fwd_bwd<<<unsigned((B + MLP_T - 1) / MLP_T), MLP_T, sm, s>>>(
      d_params, in, static_cast<const __nv_bfloat16*>(d_X), d_y, B, cw[0], cw[1], cw[2], cw[3], acts,
      pre, dels, ls);
  FR_LAUNCH_CHECK(err);
  k_mlp_wgrad<<<unsigned((L.total + 127) / 128), 128, 0, s>>>(in, B, acts, dels, d_grad);
  FR_LAUNCH_CHECK(err);
  k_sum<<<1, 256, 0, s>>>(ls, B, d_loss);
  FR_LAUNCH_CHECK(err);
  return 0;
}

}  // namespace frg
