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
// Inference and training run on the tensor cores (tcgen05, BF16 operands in shared memory, FP32
// accumulators in tensor memory): batched over elements the layers are dense [128 x 64] x [64 x 64]
// contractions, and the weight gradients [64 x 128] x [128 x 64] contractions over the samples.
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
// bound of the inference kernel's waits on its copies and MMAs (fr_tc_set_wait_limit); the drain
// after a wait that gave up always uses TC_WAIT_CYCLES, so every copy and MMA in flight completes
// before the block releases its shared and tensor memory
long long g_fwd_wait_cycles = TC_WAIT_CYCLES;
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
                                                            int8_t* __restrict__ flags, int* __restrict__ status,
                                                            long long wait_cycles) {
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
      const bool ok = tc::mbar_wait(fb[b], fphase[b], wait_cycles);
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
      const bool ok = tc::mbar_wait(mb, phase, wait_cycles);
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

// Tensor-core training: gradient of the weighted mean softmax cross-entropy over a batch.  Each
// block (one per SM: 206 KB of shared memory, all 512 tensor-memory columns) loops over tiles of
// 128 samples.  Forward as in inference, keeping every layer's input A_l in shared memory both row
// by row (the A operand of the next layer) and transposed (AT_l, the B operand of the weight
// gradient).  Backward, layer by layer from the output: the error signal dZ (BF16) is written both
// row by row (DZ, the A operand of dA = dZ W) and transposed (DZT), and one thread issues
//   dW_l += DZT * AT_{l-1}^T   (M = 128 with rows 0..63 used, K = 128 samples; accumulated in
//                               tensor memory over all the block's tiles),
//   dA_{l-1} = DZ * W_l        (B operand W_l^T, a transposed copy),
//   Z_{l-1} = A_{l-2} W_{l-1}^T  (the pre-activation recomputed instead of stored),
// after which each thread forms its row of dZ_{l-1} = dA_{l-1} * GELU'(Z_{l-1} + b).  Bias
// gradients are the row sums of DZT (thread o sums row o, in a fixed order).  Samples past the
// end of the batch get dZ = 0.  At the end the block writes its partial gradient and loss; a
// second kernel sums the blocks' partials in block order (deterministic).  Waits are bounded as
// in inference (status word, drain, free).
constexpr int TG_ROWS = 128, TG_TMEM_COLS = 512;
constexpr int TG_W1 = 0, TG_W2 = 8192, TG_W3 = 16384, TG_W4 = 24576, TG_W2T = 26624, TG_W3T = 34816,
              TG_W4T = 43008, TG_DZT = 45056, TG_A0 = 61440, TG_AT0 = 126976, TG_DZ = 192512,
              TG_BIAS = 208896, TG_MBAR = TG_BIAS + 208 * 4, TG_SMEM = TG_MBAR + 16 + 1024;
// DZT is followed by A0, which the M = 128 weight-gradient products read as rows 64..127 of their
// A operand: those rows only reach rows 64..127 of the accumulators, which are never read

__global__ void __launch_bounds__(TG_ROWS) k_mlp_grad_tc(const float* __restrict__ P, int in,
                                                         const __nv_bfloat16* __restrict__ X,
                                                         const int8_t* __restrict__ y, int64_t B, float cw0,
                                                         float cw1, float cw2, float inv_wsum,
                                                         float* __restrict__ Gp, float* __restrict__ Lp,
                                                         int* __restrict__ status) {
  extern __shared__ unsigned char sm_raw[];
  unsigned char* sm = sm_raw + ((1024 - (tc::smem_addr(sm_raw) & 1023)) & 1023);
  const int t = threadIdx.x, warp = t >> 5;
  const Lay L = lay(in);
  const int K1 = in <= 32 ? 32 : 64;
  auto put = [&](int off, uint32_t o, float v) {
    *reinterpret_cast<__nv_bfloat16*>(sm + off + o) = __float2bfloat16_rn(v);
  };
  // weights (BF16, zero padding) and their transposes for the backward products
  for (int idx = t; idx < H * 64; idx += TG_ROWS) {
    const int o = idx >> 6, k = idx & 63;
    put(TG_W1, tc::canon_off(o, k), k < in ? P[L.oW1 + o * in + k] : 0.f);
    const float w2 = P[L.oW2 + o * H + k], w3 = P[L.oW3 + o * H + k];
    put(TG_W2, tc::canon_off(o, k), w2);
    put(TG_W3, tc::canon_off(o, k), w3);
    put(TG_W2T, tc::canon_off(k, o), w2);  // W2T[i][o] = W2[o][i]
    put(TG_W3T, tc::canon_off(k, o), w3);
    if (o < 16) {
      const float w4 = o < NOUT ? P[L.oW4 + o * H + k] : 0.f;
      put(TG_W4, tc::canon_off(o, k), w4);
      put(TG_W4T, tc::canon_off_w(k, o, 16), w4);  // W4T[i][c] (16 columns)
    }
  }
  float* sb = reinterpret_cast<float*>(sm + TG_BIAS);
  for (int i = t; i < H; i += TG_ROWS) {
    sb[i] = bf16r(P[L.ob1 + i]);
    sb[H + i] = bf16r(P[L.ob2 + i]);
    sb[2 * H + i] = bf16r(P[L.ob3 + i]);
  }
  if (t < 16) sb[3 * H + t] = t < NOUT ? bf16r(P[L.ob4 + t]) : 0.f;
  const uint32_t mb = tc::smem_addr(sm + TG_MBAR);
  if (t == 0) tc::mbar_init(mb, 1);
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(sm + TG_MBAR + 8), TG_TMEM_COLS);
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(sm + TG_MBAR + 8);
  const uint32_t tlane = tmem + (uint32_t(warp * 32) << 16);
  const uint32_t ACC1 = 0, ACC2 = 64, DW[4] = {128, 192, 256, 320};  // tensor-memory columns
  const uint32_t sa = tc::smem_addr(sm);
  auto aof = [](int l) { return TG_A0 + l * 16384; };
  auto atof = [](int l) { return TG_AT0 + l * 16384; };
  const int woff[4] = {TG_W1, TG_W2, TG_W3, TG_W4};
  // one thread: D (+)= A * B^T over nk K-steps of 16, A and B tiles with the given row strides
  auto mma = [&](uint32_t dcol, int aoff, uint32_t asbo, int boff, uint32_t bsbo, int nk, int N, bool acc) {
    const uint32_t id = tc::idesc_bf16(TG_ROWS, N);
    for (int ks = 0; ks < nk; ++ks)
      tc::mma_bf16(tmem + dcol, tc::sdesc(sa + aoff + ks * 2 * tc::LBO, asbo),
                   tc::sdesc(sa + boff + ks * 2 * tc::LBO, bsbo), id, acc || ks > 0);
  };
  uint32_t phase = 0;
  bool failed = false, pend = false;
  // issue (thread 0, after the block's writes are visible to the tensor cores), commit, wait
  auto sync_issue_wait = [&](auto&& issue) -> bool {
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    if (t == 0) {
      tc::fence_after_sync();
      issue();
      tc::commit(mb);
    }
    pend = true;
    const bool ok = tc::mbar_wait(mb, phase, TC_WAIT_CYCLES);
    if (__syncthreads_or(!ok)) return false;
    phase ^= 1;
    pend = false;
    tc::fence_after_sync();
    return true;
  };
  const int64_t ntiles = (B + TG_ROWS - 1) / TG_ROWS;
  float loss = 0.f, db[4] = {0.f, 0.f, 0.f, 0.f};  // thread o: bias gradient o of each layer
  bool first = true;
  // thread t's row of dZ (FP32) -> DZ (row t) and DZT (column t), BF16; ncol columns
  auto put_dz = [&](int c, float v) {
    put(TG_DZ, tc::canon_off(t, c), v);
    put(TG_DZT, tc::canon_off_w(c, t, 128), v);
  };
  auto sum_dzt_row = [&](int o) {  // fixed-order sum over the 128 samples of row o of DZT
    float acc = 0.f;
    for (int j = 0; j < TG_ROWS; j += 8) {
      const uint4 v = *reinterpret_cast<const uint4*>(sm + TG_DZT + tc::canon_off_w(o, j, 128));
      const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 f = __bfloat1622float2(h[q]);
        acc += f.x;
        acc += f.y;
      }
    }
    return acc;
  };
  for (int64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    const int64_t row0 = tile * TG_ROWS;
    const int nrow = int(B - row0 < TG_ROWS ? B - row0 : TG_ROWS);
    const bool valid = t < nrow;
    // features: coalesced reads of the tile's contiguous rows into A0 and AT0, zero padding
    const __nv_bfloat16* xs = X + row0 * in;
    for (int idx = t; idx < TG_ROWS * in; idx += TG_ROWS) {
      const int r = idx / in, k = idx - r * in;
      const __nv_bfloat16 v = r < nrow ? xs[idx] : __float2bfloat16_rn(0.f);
      *reinterpret_cast<__nv_bfloat16*>(sm + aof(0) + tc::canon_off(r, k)) = v;
      *reinterpret_cast<__nv_bfloat16*>(sm + atof(0) + tc::canon_off_w(k, r, 128)) = v;
    }
    for (int k = in; k < 64; ++k) {
      if (k < K1) put(aof(0), tc::canon_off(t, k), 0.f);
      put(atof(0), tc::canon_off_w(k, t, 128), 0.f);
    }
    // forward: layers 1..3 into A_l / AT_l, layer 4 to logits
    for (int l = 0; l < 3 && !failed; ++l) {
      const int nk = l == 0 ? K1 / 16 : H / 16;
      if (!sync_issue_wait([&] { mma(ACC1, aof(l), tc::SBO, woff[l], tc::SBO, nk, H, false); })) {
        failed = true;
        break;
      }
      const float* bl = sb + H * l;
#pragma unroll
      for (int c0 = 0; c0 < H; c0 += 16) {
        uint32_t r[16];
        tc::tmem_ld16(tlane + ACC1 + uint32_t(c0), r);
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float a = gelu(__uint_as_float(r[j]) + bl[c0 + j]);
          put(aof(l + 1), tc::canon_off(t, c0 + j), a);
          put(atof(l + 1), tc::canon_off_w(c0 + j, t, 128), a);
        }
      }
    }
    if (failed) break;
    if (!sync_issue_wait([&] { mma(ACC1, aof(3), tc::SBO, TG_W4, tc::SBO, H / 16, 16, false); })) {
      failed = true;
      break;
    }
    {
      uint32_t r[16];
      tc::tmem_ld16(tlane + ACC1, r);
      tc::tmem_wait_ld();
      float dz[NOUT] = {0.f, 0.f, 0.f};
      if (valid) {
        float o[NOUT];
#pragma unroll
        for (int c = 0; c < NOUT; ++c) o[c] = __uint_as_float(r[c]) + sb[3 * H + c];
        const int cls = int(y[row0 + t]) + 1;
        const float w = cls == 0 ? cw0 : (cls == 1 ? cw1 : cw2);
        const float mx = fmaxf(o[0], fmaxf(o[1], o[2]));
        const float e0 = expf(o[0] - mx), e1 = expf(o[1] - mx), e2 = expf(o[2] - mx);
        const float sum = e0 + e1 + e2;
        const float pz[NOUT] = {e0 / sum, e1 / sum, e2 / sum};
        loss += -w * inv_wsum * logf(pz[cls]);
#pragma unroll
        for (int c = 0; c < NOUT; ++c) dz[c] = w * inv_wsum * (pz[c] - (c == cls ? 1.f : 0.f));
      }
      for (int c = 0; c < 16; ++c) put(TG_DZ, tc::canon_off(t, c), c < NOUT ? dz[c] : 0.f);
      for (int c = 0; c < NOUT; ++c) put(TG_DZT, tc::canon_off_w(c, t, 128), dz[c]);
    }
    // backward: l = 3 (output layer's weights) down to 0
    for (int l = 3; l >= 0 && !failed; --l) {
      // dW_l += DZT * AT_{l-1}; for l > 0 also dA = DZ * W_l and the recomputed Z of layer l-1
      const bool ok = sync_issue_wait([&] {
        mma(DW[l], TG_DZT, 2048, atof(l), 2048, TG_ROWS / 16, H, !first);
        if (l > 0) {
          if (l == 3)
            mma(ACC1, TG_DZ, tc::SBO, TG_W4T, 256, 1, H, false);
          else
            mma(ACC1, TG_DZ, tc::SBO, l == 2 ? TG_W3T : TG_W2T, tc::SBO, H / 16, H, false);
          mma(ACC2, aof(l - 1), tc::SBO, woff[l - 1], tc::SBO, l - 1 == 0 ? K1 / 16 : H / 16, H, false);
        }
      });
      // bias gradient of layer l from the DZT rows the products above read (no writes yet)
      if (t < (l == 3 ? NOUT : H)) db[l] += sum_dzt_row(t);
      if (!ok) {
        failed = true;
        break;
      }
      if (l == 0) break;
      __syncthreads();  // every row of DZT summed before it is overwritten
      // dZ of layer l-1: dA * GELU'(Z + b)
      const float* bl = sb + H * (l - 1);
#pragma unroll
      for (int c0 = 0; c0 < H; c0 += 16) {
        uint32_t ra[16], rz[16];
        tc::tmem_ld16(tlane + ACC1 + uint32_t(c0), ra);
        tc::tmem_ld16(tlane + ACC2 + uint32_t(c0), rz);
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float d = valid ? __uint_as_float(ra[j]) * gelu_d(__uint_as_float(rz[j]) + bl[c0 + j]) : 0.f;
          put_dz(c0 + j, d);
        }
      }
    }
    first = false;
  }
  if (failed) {
    if (t == 0) atomicExch(status, 1);
    if (pend) tc::mbar_wait(mb, phase, TC_WAIT_CYCLES);
  }
  __syncthreads();
  // the block's partial gradient in the parameter layout, and its loss
  float* g = Gp + int64_t(blockIdx.x) * L.total;
  if (warp < 2) {  // rows 0..63 of the weight-gradient accumulators (tensor-memory lanes 0..63)
    tc::fence_after_sync();
    for (int l = 0; l < 4; ++l) {
      const int nin = l == 0 ? in : H, ow = l == 0 ? L.oW1 : l == 1 ? L.oW2 : l == 2 ? L.oW3 : L.oW4;
      const int nout = l == 3 ? NOUT : H;
#pragma unroll
      for (int c0 = 0; c0 < H; c0 += 16) {
        uint32_t r[16];
        tc::tmem_ld16(tlane + DW[l] + uint32_t(c0), r);
        tc::tmem_wait_ld();
        if (t < nout && !first)
          for (int j = 0; j < 16; ++j)
            if (c0 + j < nin) g[ow + t * nin + c0 + j] = __uint_as_float(r[j]);
      }
    }
  }
  if (first) {  // a block without tiles contributes zeros
    for (int k = t; k < L.total; k += TG_ROWS) g[k] = 0.f;
  } else {
    if (t < H) {
      g[L.ob1 + t] = db[0];
      g[L.ob2 + t] = db[1];
      g[L.ob3 + t] = db[2];
    }
    if (t < NOUT) g[L.ob4 + t] = db[3];
  }
  // loss: warp sums, then the four warps in order
  float* red = reinterpret_cast<float*>(sm + TG_BIAS);
  __syncthreads();
#pragma unroll
  for (int w = 16; w > 0; w >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, w);
  if ((t & 31) == 0) red[warp] = loss;
  __syncthreads();
  if (t == 0) Lp[blockIdx.x] = red[0] + red[1] + red[2] + red[3];
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_free(tmem, TG_TMEM_COLS);
  }
}

// sums of the blocks' partial gradients and losses, in block order
__global__ void k_grad_reduce(const float* __restrict__ Gp, const float* __restrict__ Lp, int nblk, int total,
                              float* __restrict__ G, float* __restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < total) {
    float a = 0.f;
    for (int c = 0; c < nblk; ++c) a += Gp[int64_t(c) * total + p];
    G[p] = a;
  }
  if (p == 0 && loss) {
    float a = 0.f;
    for (int c = 0; c < nblk; ++c) a += Lp[c];
    *loss = a;
  }
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

}  // namespace

int mlp_param_count(int in) { return lay(in).total; }

void mlp_set_wait_cycles(long long cycles) { g_fwd_wait_cycles = cycles > 0 ? cycles : TC_WAIT_CYCLES; }

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
                                               d_logits, d_flags, d_status, g_fwd_wait_cycles);
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

// gradient (into G, total floats) and loss of one batch on the tensor cores; *d_st (scratch)
// becomes nonzero if a completion wait gave up
static int grad_tc(const float* d_params, int in, const void* d_X, const int8_t* d_y, int64_t B,
                   const float* cw, float* G, float* d_loss, Scratch& S, int** d_st, cudaStream_t s, Err* err) {
  if (B <= 0) return set_error(err, FR_EINVAL, "empty batch");
  if (in < 1 || in > 64) return set_error(err, FR_EINVAL, "the MLP takes 1..64 inputs");
  const Lay L = lay(in);
  int dev = 0, sms = 0;
  FR_CUDA(err, cudaGetDevice(&dev));
  FR_CUDA(err, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t ntiles = (B + TG_ROWS - 1) / TG_ROWS;
  const int grid = int(ntiles < sms ? ntiles : sms);  // one block per SM (shared memory, TMEM)
  float* Gp = S.get<float>(size_t(grid) * L.total);
  float* Lp = S.get<float>(size_t(grid));
  int* st = S.get<int>(1);
  if (!Gp || !Lp || !st) return set_error(err, FR_ENOMEM, "training scratch");
  FR_CUDA(err, cudaMemsetAsync(st, 0, 4, s));
  FR_CUDA(err, cudaFuncSetAttribute(k_mlp_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TG_SMEM));
  // class weights normalised by the batch's total weight: cw[0..2], and cw[3] = 1 / sum_b w_{y_b}
  k_mlp_grad_tc<<<unsigned(grid), TG_ROWS, TG_SMEM, s>>>(d_params, in, static_cast<const __nv_bfloat16*>(d_X),
                                                         d_y, B, cw[0], cw[1], cw[2], cw[3], Gp, Lp, st);
  FR_LAUNCH_CHECK(err);
  k_grad_reduce<<<unsigned((L.total + 255) / 256), 256, 0, s>>>(Gp, Lp, grid, L.total, G, d_loss);
  FR_LAUNCH_CHECK(err);
  *d_st = st;
  return 0;
}

static int check_status(const int* d_st, cudaStream_t s, Err* err) {
  int h = 0;
  FR_CUDA(err, cudaMemcpyAsync(&h, d_st, 4, cudaMemcpyDeviceToHost, s));
  FR_CUDA(err, cudaStreamSynchronize(s));
  return h ? set_error(err, FR_ETIMEOUT, "a tensor-core completion wait gave up (training)") : 0;
}

int mlp_train_step(float* d_params, float* d_m, float* d_v, int64_t step, int in, const void* d_X,
                   const int8_t* d_y, int64_t B, const float* cw, float lr, float* d_loss,
                   Alloc& A, cudaStream_t s, Err* err) {
  const Lay L = lay(in);
  Scratch S(&A);
  float* G = S.get<float>(L.total);
  if (!G) return set_error(err, FR_ENOMEM, "training scratch");
  int* st = nullptr;
  FR_TRY(grad_tc(d_params, in, d_X, d_y, B, cw, G, d_loss, S, &st, s, err));
  const float b1 = 0.9f, b2 = 0.999f;
  float c1 = 1.f - std::pow(b1, float(step + 1)), c2 = 1.f - std::pow(b2, float(step + 1));
  k_adam<<<unsigned((L.total + 255) / 256), 256, 0, s>>>(d_params, d_m, d_v, G, L.total, lr, b1, b2,
                                                         1e-8f, c1, c2);
  FR_LAUNCH_CHECK(err);
  return check_status(st, s, err);
}

int mlp_grad(const float* d_params, int in, const void* d_X, const int8_t* d_y, int64_t B,
             const float* cw, float* d_grad, float* d_loss, Alloc& A, cudaStream_t s, Err* err) {
  Scratch S(&A);
  int* st = nullptr;
  FR_TRY(grad_tc(d_params, in, d_X, d_y, B, cw, d_grad, d_loss, S, &st, s, err));
  return check_status(st, s, err);
}

}  // namespace frg
