// fr_tc_stage.cu -- element stage of the tensor-core operator forms (fr_config.precision 2: TF32,
// 3: split BF16 "bf16x3"), 3D p = 3 (64 Gauss-Legendre points per hexahedron).
//
// The volume part of the corrected-flux derivative of Sec. 2.1, sum_a sum_j Dt_ij f_a,j with the
// correction folded into the 1D operator Dt, is a contraction over the element's points.  Here it
// runs on the fifth-generation tensor cores (tcgen05.mma, FP32 accumulation in tensor memory); the
// fluxes, the correction terms, the Runge-Kutta combination (FP64) and the traces of the new state
// run on the CUDA cores as in the FP32 form.
//
// Per block: 25 elements, 256 threads.  Rows of the MMA are (element, variable) pairs (125 of 128
// rows used).  For each axis a the fluxes f_a of the block form the A operand (128 rows x 64
// points, K-major, no swizzle), and the 64 points are taken in blocks of 16:
//   x: natural point order p = x + 4y + 16z; a block is one z-plane and the 16 x 16 operator is
//      B_x[(x,y)][(x',y')] = delta(y,y') Dt[x][x'];
//   y: the same blocks, B_y[(x,y)][(x',y')] = delta(x,x') Dt[y][y'], accumulated onto x;
//   z: the points re-ordered z-fastest, c = z + 4x + 16y, so that a block of 16 holds four whole
//      z-lines and B_x applies along z; accumulated in a second tensor-memory region.
// So one M = 128, N = 16, K = 16 product per block and axis (bf16x3: three, hi*hi + hi*lo + lo*hi;
// TF32: two of K = 8), 12 blocks per element tile, D in 128 tensor-memory columns.
//
// Accuracy.  The tensor cores see f - f_ref with f_ref the flux at the element's first point (per
// axis and variable): constants are removed before rounding, so a uniform flow gives exactly zero.
// The folded operator maps a constant c to -(g'_L + g'_R) c, so the removed part returns through
// the correction terms: R_i = (Dt (f - f_ref))_i + gLh_i (2F_L - 2 f_ref) + gRh_i (2F_R - 2 f_ref)
// (the interface kernel stores twice the common flux, the slopes carry the 1/2), exact in real
// arithmetic and evaluated in FP32.
//
// Waits on the MMA completions are bounded (about a second of clock cycles); on expiry the block
// records FR_ETIMEOUT in the status word, waits once more (bounded) for its MMAs in flight, frees
// its tensor memory and exits without writing its elements.
#include <cuda_bf16.h>

#include <cstring>

#include "fr_kernels.cuh"
#include "fr_tc.cuh"

namespace frg {
namespace {

constexpr int TS_E = 25;                  // elements per block
constexpr int TS_T = 256;                 // threads per block
constexpr int TS_N = 64, TS_NV = 5, TS_NF = 16;
constexpr int TS_EU = TS_NV * TS_N;       // 320 values per element state
constexpr int TS_EF = 6 * TS_NV * TS_NF;  // 480 face values per element
constexpr int TS_RS = 65;                 // padded row stride of the staged volume sums (floats)
constexpr uint32_t TS_TMEM_COLS = 128;    // D_xy: columns 0..63, D_z: 64..127
constexpr long long TS_WAIT_CYCLES = 2000000000ll;

// shared memory (bytes from a 1024-aligned base)
constexpr int OFF_A = 0;                        // A operand of one axis / staged volume sums
constexpr int SZ_A = 32768;                     // 128 x 64 x (2 + 2 B or 4 B); 125 x 65 x 4 = 32500
constexpr int OFF_B = OFF_A + SZ_A;             // B_x, B_y (bf16: hi, lo each 512 B; tf32: 1 KB each)
constexpr int SZ_B = 2048;
constexpr int OFF_U = OFF_B + SZ_B;             // stage state, float [25][5][64], later the new state
constexpr int SZ_U = TS_E * TS_EU * 4;
constexpr int OFF_REF = OFF_U + SZ_U;           // reference fluxes, float [25][3][5]
constexpr int SZ_REF = 1504;
constexpr int OFF_H2 = OFF_REF + SZ_REF;        // per element c * (-2/h), double [25]
constexpr int OFF_BAR = OFF_H2 + TS_E * 8;      // mbarrier (8 B), tensor-memory base (4 B)
constexpr int SMEM_USED = OFF_BAR + 16;
constexpr int SMEM_BYTES = SMEM_USED + 1024;    // + alignment slack
static_assert(TS_E * TS_NV * TS_RS * 4 <= SZ_A, "staged sums must fit the A region");

// B operands as 32-bit words in their shared-memory layout, prepared on the host: for bf16x3 the
// 2 x 2 x 16 x 16 BF16 values (B_x hi, B_x lo, B_y hi, B_y lo) packed in pairs; for TF32 the
// 2 x 16 x 16 values rounded to TF32.
struct TcB {
  uint32_t w[512];
};

// byte offset of (r, k) in a K-major no-swizzle tile of `cols` columns of `esz`-byte elements
// (core matrices of 8 rows x 16 bytes; 16 bytes along K per core matrix, 128 bytes between core
// matrices along K, 8-row groups cols*esz*8/... apart)
__host__ __device__ constexpr uint32_t kmaj_off(int r, int k, int cols, int esz) {
  return uint32_t((r >> 3) * (cols * esz * 8) + ((k * esz) >> 4) * 128 + (r & 7) * 16 + ((k * esz) & 15));
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// D[M x N] (+)= A * B^T of kind::tf32 (K = 8 per instruction), issued by one thread
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, bool acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(uint32_t(acc))
      : "memory");
}
// instruction descriptor of kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9, 10-12 = 2),
// both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}
__device__ __forceinline__ uint64_t sdesc_sbo(uint32_t addr, uint32_t sbo) { return tc::sdesc(addr, sbo); }

// pointwise Euler flux along `axis` of the state q (5 values), FP32
__device__ __forceinline__ void euler_flux(const float* q, int axis, float gm1, float ngmh, float* f) {
  const float rinv = __fdividef(1.0f, q[0]);
  const float vx = q[1] * rinv, vy = q[2] * rinv, vz = q[3] * rinv;
  const float m2 = fmaf(q[1], vx, fmaf(q[2], vy, q[3] * vz));
  const float p = fmaf(ngmh, m2, gm1 * q[4]);
  const float va = axis == 0 ? vx : axis == 1 ? vy : vz;
  f[0] = q[1 + axis];
  f[1] = q[1] * va + (axis == 0 ? p : 0.f);
  f[2] = q[2] * va + (axis == 1 ? p : 0.f);
  f[3] = q[3] * va + (axis == 2 ? p : 0.f);
  f[4] = (q[4] + p) * va;
}

// A-operand column of point p = x + 4y + 16z for axis `axis`
__device__ __forceinline__ int a_col(int axis, int p) {
  if (axis < 2) return p;
  const int x = p & 3, y = (p >> 2) & 3, z = p >> 4;
  return z + 4 * x + 16 * y;
}

// the volume sums of one row (element, variable) for the natural points 32H .. 32H+31, from
// tensor memory (warp-collective: every lane of the warp takes part) into dst (null: row absent):
// D_xy columns 32H.., plus D_z where column c = z + 4x + 16y holds natural point x + 4y + 16z
template <int H>
__device__ __forceinline__ void drain_row(uint32_t tl, float* dst) {
  float R[32];
  uint32_t v[16];
  tc::tmem_ld16(tl + uint32_t(32 * H), v);
  tc::tmem_wait_ld();
#pragma unroll
  for (int j = 0; j < 16; ++j) R[j] = __uint_as_float(v[j]);
  tc::tmem_ld16(tl + uint32_t(32 * H + 16), v);
  tc::tmem_wait_ld();
#pragma unroll
  for (int j = 0; j < 16; ++j) R[16 + j] = __uint_as_float(v[j]);
#pragma unroll
  for (int y = 0; y < 4; ++y) {
    tc::tmem_ld16(tl + uint32_t(64 + 16 * y), v);
    tc::tmem_wait_ld();
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int dz = 0; dz < 2; ++dz) R[x + 4 * y + 16 * dz] += __uint_as_float(v[(2 * H + dz) + 4 * x]);
  }
  if (dst) {
#pragma unroll
    for (int j = 0; j < 32; ++j) dst[32 * H + j] = R[j];
  }
}

template <int KIND>  // 0: TF32, 1: bf16x3
__global__ void __launch_bounds__(TS_T) k_stage_tc(StageArgs A, const __grid_constant__ OpsT<float> ops,
                                                   const __grid_constant__ TcB tb) {
  int* status = A.status;
  extern __shared__ unsigned char sm_raw[];
  unsigned char* sm = sm_raw + ((1024 - (tc::smem_addr(sm_raw) & 1023)) & 1023);
  float* su = reinterpret_cast<float*>(sm + OFF_U);
  float* sref = reinterpret_cast<float*>(sm + OFF_REF);
  double* sh2 = reinterpret_cast<double*>(sm + OFF_H2);
  const uint32_t mb = tc::smem_addr(sm + OFF_BAR);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t e0 = int64_t(blockIdx.x) * TS_E;
  const int ne = int((A.M - e0) < TS_E ? (A.M - e0) : TS_E);
  const float gm1 = ops.gm1, ngmh = ops.ngmh;
  if (tid == 0) tc::mbar_init(mb, 1);
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(sm + OFF_BAR + 8), TS_TMEM_COLS);
  // B operands (prepared on the host in their shared-memory layout)
  for (int k = tid; k < 512; k += TS_T) reinterpret_cast<uint32_t*>(sm + OFF_B)[k] = tb.w[k];
  // the stage state and the keys are final before the interface kernel this one depends on
  // started: they are read, and the whole volume contraction done, before the wait on it
  for (int k = tid; k < ne * TS_EU; k += TS_T) su[k] = Ar<float>::from_d(A.us[e0 * TS_EU + k]);
  if (tid < ne) sh2[tid] = -A.c * (double(1ull << A.g.depth(A.keys[e0 + tid])) * A.twoL);
  __syncthreads();
  if (tid < ne * 3) {  // reference fluxes: the flux at the element's first point
    const int e = tid / 3, a = tid % 3;
    float q[5], f[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) q[v] = su[e * TS_EU + v * TS_N];
    euler_flux(q, a, gm1, ngmh, f);
#pragma unroll
    for (int v = 0; v < 5; ++v) sref[(e * 3 + a) * 5 + v] = f[v];
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(sm + OFF_BAR + 8);
  const uint32_t sA = tc::smem_addr(sm + OFF_A), sB = tc::smem_addr(sm + OFF_B);
  bool failed = false, mma_pend = false;
  uint32_t phase = 0;
  for (int a = 0; a < 3 && !failed; ++a) {
    // fluxes of axis a minus the reference, into the A operand; rows of absent elements are zero
    for (int t = tid; t < TS_E * TS_N; t += TS_T) {
      const int e = t >> 6, p = t & 63;
      float f[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      if (e < ne) {
        float q[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) q[v] = su[e * TS_EU + v * TS_N + p];
        euler_flux(q, a, gm1, ngmh, f);
#pragma unroll
        for (int v = 0; v < 5; ++v) f[v] -= sref[(e * 3 + a) * 5 + v];
      }
      const int c = a_col(a, p);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const int r = e * 5 + v;
        if (KIND == 1) {
          const __nv_bfloat16 hi = __float2bfloat16_rn(f[v]);
          const __nv_bfloat16 lo = __float2bfloat16_rn(f[v] - __bfloat162float(hi));
          *reinterpret_cast<__nv_bfloat16*>(sm + OFF_A + kmaj_off(r, c, 64, 2)) = hi;
          *reinterpret_cast<__nv_bfloat16*>(sm + OFF_A + 16384 + kmaj_off(r, c, 64, 2)) = lo;
        } else {
          *reinterpret_cast<uint32_t*>(sm + OFF_A + kmaj_off(r, c, 64, 4)) = tf32_rna(f[v]);
        }
      }
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t d0 = tmem + (a == 2 ? 64u : 0u);
      const bool acc0 = a == 1;  // y accumulates onto x; x and z start their regions
      for (int kb = 0; kb < 4; ++kb) {
        const uint32_t d = d0 + uint32_t(16 * kb);
        if (KIND == 1) {
          const uint32_t id = tc::idesc_bf16(128, 16);
          const uint32_t bhi = sB + (a == 1 ? 1024u : 0u), blo = bhi + 512u;
          const uint64_t ahi = sdesc_sbo(sA + uint32_t(kb * 256), 1024), alo = sdesc_sbo(sA + 16384u + uint32_t(kb * 256), 1024);
          tc::mma_bf16(d, ahi, sdesc_sbo(bhi, 256), id, acc0);
          tc::mma_bf16(d, ahi, sdesc_sbo(blo, 256), id, true);
          tc::mma_bf16(d, alo, sdesc_sbo(bhi, 256), id, true);
        } else {
          const uint32_t id = idesc_tf32(128, 16);
          const uint32_t bb = sB + (a == 1 ? 1024u : 0u);
          mma_tf32(d, sdesc_sbo(sA + uint32_t(kb * 512), 2048), sdesc_sbo(bb, 512), id, acc0);
          mma_tf32(d, sdesc_sbo(sA + uint32_t(kb * 512 + 256), 2048), sdesc_sbo(bb + 256u, 512), id, true);
        }
      }
      tc::commit(mb);
    }
    mma_pend = true;
    const bool ok = tc::mbar_wait(mb, phase, TS_WAIT_CYCLES);
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    phase ^= 1;
    mma_pend = false;
    tc::fence_after_sync();
  }
  if (failed) {
    pdl_wait_then_release();  // global writes come after the wait on the preceding kernel
    if (tid == 0) atomicExch(status, 1);
    if (mma_pend) tc::mbar_wait(mb, phase, TS_WAIT_CYCLES);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
      tc::fence_after_sync();
      tc::tmem_free(tmem, TS_TMEM_COLS);
    }
    return;
  }
  // volume sums out of tensor memory into shared memory, one row (element, variable) per lane;
  // warps w and w + 4 read the same 32 lanes, for the points 0..31 and 32..63
  {
    const int qd = warp & 3, r = 32 * qd + lane;
    const uint32_t tl = tmem + (uint32_t(32 * qd) << 16);
    float* dst = r < ne * 5 ? reinterpret_cast<float*>(sm + OFF_A) + r * TS_RS : nullptr;
    if (warp < 4)
      drain_row<0>(tl, dst);
    else
      drain_row<1>(tl, dst);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_free(tmem, TS_TMEM_COLS);
  }
  // the common fluxes come from the interface kernel: wait for it
  pdl_wait_then_release();
  const float* fcomm = static_cast<const float*>(A.fcomm);
  const float* sR = reinterpret_cast<const float*>(sm + OFF_A);
  for (int t = tid; t < ne * TS_N; t += TS_T) {
    const int e = t >> 6, i = t & 63;
    float R[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) R[v] = sR[(e * 5 + v) * TS_RS + i];
    const float* fe = fcomm + (e0 + e) * TS_EF;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      int qf, ia;
      pt_split<3, 4>(i, a, &qf, &ia);
      const float* Fm = fe + (2 * a) * TS_NV * TS_NF + qf;
      const float* Fp = fe + (2 * a + 1) * TS_NV * TS_NF + qf;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const float r2 = 2.0f * sref[(e * 3 + a) * 5 + v];
        R[v] = fmaf(ops.gLh[ia], Fm[v * TS_NF] - r2, fmaf(ops.gRh[ia], Fp[v * TS_NF] - r2, R[v]));
      }
    }
    const double cs = sh2[e];
    const int64_t base = (e0 + e) * TS_EU + i;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const double us = A.us[base + v * TS_N];
      double o = fma(cs, Ar<float>::to_d(R[v]), (A.rk & RK_B1) ? us : A.b * us);
      if (A.rk & RK_A) o = fma(A.a, A.un[base + v * TS_N], o);
      A.out[base + v * TS_N] = o;
      su[e * TS_EU + v * TS_N + i] = Ar<float>::from_d(o);
    }
  }
  __syncthreads();
  float* trace_out = static_cast<float*>(A.trace_out);
  if (trace_out) {
    // one thread per (element, face, face point), all variables from one set of indices
    for (int k = tid; k < ne * 6 * TS_NF; k += TS_T) {
      const int le = k / (6 * TS_NF), r = k % (6 * TS_NF);
      const int f = r / TS_NF, qq = r % TS_NF;
      const float* lf = (f & 1) ? ops.lp : ops.lm;
      int pts[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) pts[j] = line_pt<3, 4>(f >> 1, qq, j);
      float* to = trace_out + (e0 + le) * TS_EF + f * TS_NV * TS_NF + qq;
#pragma unroll
      for (int v = 0; v < TS_NV; ++v) {
        const float* ue = su + le * TS_EU + v * TS_N;
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) s = fmaf(lf[j], ue[pts[j]], s);
        to[v * TS_NF] = s;
      }
    }
  }
}

// ---- host side ----
uint16_t bf16_bits_rn(float x) {  // round to nearest even (finite inputs)
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return uint16_t(u >> 16);
}
float bf16_to_float(uint16_t b) {
  uint32_t u = uint32_t(b) << 16;
  float x;
  std::memcpy(&x, &u, 4);
  return x;
}
uint32_t tf32_bits_rn(float x) {  // round to nearest (ties away), low 13 bits cleared
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u += 0x1000u;
  return u & ~0x1FFFu;
}

TcB make_tc_b(int kind, const DevOps& o) {
  TcB b{};
  unsigned char* bytes = reinterpret_cast<unsigned char*>(b.w);
  for (int which = 0; which < 2; ++which)
    for (int n = 0; n < 16; ++n)
      for (int k = 0; k < 16; ++k) {
        const int xn = n & 3, yn = n >> 2, xk = k & 3, yk = k >> 2;
        const double d = which == 0 ? (yn == yk ? o.Dt[xn][xk] : 0.0) : (xn == xk ? o.Dt[yn][yk] : 0.0);
        if (kind == 1) {
          const uint16_t hi = bf16_bits_rn(float(d));
          const uint16_t lo = bf16_bits_rn(float(d - double(bf16_to_float(hi))));
          const uint32_t off = kmaj_off(n, k, 16, 2);
          std::memcpy(bytes + which * 1024 + off, &hi, 2);
          std::memcpy(bytes + which * 1024 + 512 + off, &lo, 2);
        } else {
          const uint32_t t = tf32_bits_rn(float(d));
          std::memcpy(bytes + which * 1024 + kmaj_off(n, k, 16, 4), &t, 4);
        }
      }
  return b;
}

template <int KIND>
int launch_tc(const StageArgs& A, const DevOps& o, cudaStream_t s, Err* err) {
  static bool attr = false;
  if (!attr) {
    FR_CUDA(err, cudaFuncSetAttribute(k_stage_tc<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    attr = true;
  }
  OpsT<float> ops = make_ops_t<float>(o);
  set_gas(&ops, A.gamma);
  const TcB tb = make_tc_b(KIND, o);
  const unsigned nb = unsigned((A.M + TS_E - 1) / TS_E);
  if (launch_dependent_smem(k_stage_tc<KIND>, nb, TS_T, size_t(SMEM_BYTES), s, A, ops, tb) != cudaSuccess)
    return set_error(err, FR_ECUDA, "tensor-core element kernel launch");
  FR_LAUNCH_CHECK(err);
  return 0;
}

}  // namespace

int launch_stage_tc(int prec, int dim, int p, const StageArgs& A, const DevOps& o, cudaStream_t s, Err* err) {
  if (dim != 3 || p != 3) return set_error(err, FR_EINVAL, "tensor-core operator forms are built for 3D p = 3");
  if (!A.status) return set_error(err, FR_EINVAL, "tensor-core element kernel needs a status word");
  if (A.M <= 0) return 0;
  return prec == 2 ? launch_tc<0>(A, o, s, err) : launch_tc<1>(A, o, s, err);
}

}  // namespace frg
