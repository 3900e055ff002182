// fr_kernels.cuh -- the time-step kernels of flux reconstruction (arXiv 2306.06744, Sec. 2.1 and
// 4.3), templated on the dimension, the number of points per direction n = p+1 and the
// arithmetic type T (double, float or double-word ff; see fr_arith.cuh).  The state u is FP64 in
// memory for every T; face traces and common fluxes are stored in T.  Each precision is
// instantiated in its own translation unit (fr_prec_*.cu).
#pragma once

#include <type_traits>

#include "fr_arith.cuh"
#include "fr_internal.cuh"
#include "fr_solver.cuh"

namespace frg {

// Operator tables in the arithmetic type (passed by value: constant bank)
template <class T>
struct OpsT {
  T Dt[NPMAX][NPMAX];
  T D[NPMAX][NPMAX];  // plain derivative l_j'(x_i) (density-gradient indicator)
  // gLh, gRh: half the correction slopes g'_L, g'_R at the solution points, because the
  // interface kernel stores twice the common flux (exact scalings by 2 and 1/2)
  T gLh[NPMAX], gRh[NPMAX], lm[NPMAX], lp[NPMAX];
  T I[2][NPMAX][NPMAX];
  T P[2][NPMAX][NPMAX];
  // gas constants in the arithmetic type, formed on the host (set_gas): gamma, gamma - 1 and
  // -(gamma - 1)/2, so that no thread spends FP64 operations on them
  T gam, gm1, ngmh;
};

inline double host_conv(double x, double*) { return x; }
inline float host_conv(double x, float*) { return float(x); }
inline ff host_conv(double x, ff*) {
  float h = float(x);
  float l = float(x - double(h));
  return ff{h, l};
}

template <class T>
void set_gas(OpsT<T>* r, double gamma) {
  T* tag = nullptr;
  r->gam = host_conv(gamma, tag);
  r->gm1 = host_conv(gamma - 1.0, tag);
  r->ngmh = host_conv(-0.5 * (gamma - 1.0), tag);
}

template <class T>
OpsT<T> make_ops_t(const DevOps& o) {
  OpsT<T> r{};
  T* tag = nullptr;
  for (int i = 0; i < NPMAX; ++i) {
    r.gLh[i] = host_conv(0.5 * o.gL[i], tag);
    r.gRh[i] = host_conv(0.5 * o.gR[i], tag);
    r.lm[i] = host_conv(o.lm[i], tag);
    r.lp[i] = host_conv(o.lp[i], tag);
    for (int j = 0; j < NPMAX; ++j) {
      r.Dt[i][j] = host_conv(o.Dt[i][j], tag);
      r.D[i][j] = host_conv(o.D[i][j], tag);
      for (int h = 0; h < 2; ++h) {
        r.I[h][i][j] = host_conv(o.I[h][i][j], tag);
        r.P[h][i][j] = host_conv(o.P[h][i][j], tag);
      }
    }
  }
  return r;
}

template <int DIM, int NP>
struct Sz {
  static constexpr int N = DIM == 2 ? NP * NP : NP * NP * NP;
  static constexpr int NF = DIM == 2 ? NP : NP * NP;
  static constexpr int NV = DIM + 2;
  static constexpr int NFC = 2 * DIM;
  static constexpr int NSUB = 1 << (DIM - 1);
  static constexpr int EU = NV * N;         // values per element state
  static constexpr int EF = NFC * NV * NF;  // values per element face data
  // elements per block of the element kernel, one thread per point: 128/N elements, except for
  // N = 27 (3D, p = 2) where 4 elements would leave 20 of 128 threads idle: 7 elements fill
  // 189 of 192 (the shared-memory stage stays under 48 KB)
  static constexpr int EPB = N == 27 ? 7 : ((128 / N) > 0 ? (128 / N) : 1);
  static constexpr int BT = (EPB * N + 31) / 32 * 32;  // threads per block
};

// element point index of position j along `axis` on the line through face point q
template <int DIM, int NP>
__device__ __forceinline__ int line_pt(int axis, int q, int j) {
  if (DIM == 2) return axis == 0 ? j + NP * q : q + NP * j;
  if (axis == 0) return j + NP * q;
  if (axis == 1) return (q % NP) + NP * j + NP * NP * (q / NP);
  return q + NP * NP * j;
}
// face point index on the face of `axis` for element point i, and i's position along the axis
template <int DIM, int NP>
__device__ __forceinline__ void pt_split(int i, int axis, int* q, int* ia) {
  int ix = i % NP, iy = (i / NP) % NP, iz = DIM == 3 ? i / (NP * NP) : 0;
  if (axis == 0) {
    *ia = ix;
    *q = DIM == 2 ? iy : iy + NP * iz;
  } else if (axis == 1) {
    *ia = iy;
    *q = DIM == 2 ? ix : ix + NP * iz;
  } else {
    *ia = iz;
    *q = ix + NP * iy;
  }
}

// Twice the Rusanov common flux along +axis between the minus-side state qL and the plus-side
// qR, F2 = f(qL) + f(qR) - lambda (qR - qL) with lambda = max(|u_n| + c) of the two states
// (Sec. 4.3); the factor 1/2 is carried by the correction slopes.  ngmh = -(gamma - 1)/2, so
// that p = (gamma - 1) E + ngmh |m|^2 / rho.
template <int DIM, class T>
__device__ __forceinline__ void rusanov2_t(const T* qL, const T* qR, int axis, T gam, T gm1, T ngmh,
                                           T* F2) {
  constexpr int NV = DIM + 2;
  // both reciprocal densities from one reciprocal: 1/rho_L = rho_R / (rho_L rho_R), and so on
  const T rLR = rcp_t(qL[0] * qR[0]);
  T rL = qR[0] * rLR, rR = qL[0] * rLR;
  T m2L = qL[1] * qL[1], m2R = qR[1] * qR[1];
#pragma unroll
  for (int b = 1; b < DIM; ++b) {
    m2L = fma_t(qL[1 + b], qL[1 + b], m2L);
    m2R = fma_t(qR[1 + b], qR[1 + b], m2R);
  }
  T pL = fma_t(ngmh, m2L * rL, gm1 * qL[NV - 1]);
  T pR = fma_t(ngmh, m2R * rR, gm1 * qR[NV - 1]);
  // normal momenta, selected with unrolled predicates so the state stays in registers
  T mnL = qL[1], mnR = qR[1];
#pragma unroll
  for (int b = 1; b < DIM; ++b)
    if (b == axis) {
      mnL = qL[1 + b];
      mnR = qR[1 + b];
    }
  T vL = mnL * rL, vR = mnR * rR;
  T cL = sqrt_t(gam * pL * rL), cR = sqrt_t(gam * pR * rR);
  T lam = fmax_t(fabs_t(vL) + cL, fabs_t(vR) + cR);
  T fL[NV], fR[NV];
  fL[0] = mnL;
  fR[0] = mnR;
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    T a = qL[1 + b] * vL, c = qR[1 + b] * vR;
    fL[1 + b] = (b == axis) ? a + pL : a;
    fR[1 + b] = (b == axis) ? c + pR : c;
  }
  fL[NV - 1] = (qL[NV - 1] + pL) * vL;
  fR[NV - 1] = (qR[NV - 1] + pR) * vR;
#pragma unroll
  for (int v = 0; v < NV; ++v) F2[v] = fma_t(lam, qL[v] - qR[v], fL[v] + fR[v]);
}

// traces tr[e][f][v][q] = sum_j l_j(+-1) u[e][v][line point j]  (mortar procedure step 1).
// Blocks of EPB elements as in the element kernel: the elements' state is staged in shared memory
// with coalesced loads, then one thread per (element, face, face point) forms all variables.
template <int DIM, int NP, class T>
__global__ void __launch_bounds__(Sz<DIM, NP>::BT) k_traces_t(const double* __restrict__ u, int64_t M,
                                                              const __grid_constant__ OpsT<T> ops,
                                                              T* __restrict__ tr, const int8_t* __restrict__ mask,
                                                              const int64_t* __restrict__ d_M) {
  pdl_wait_then_release();
  using S = Sz<DIM, NP>;
  constexpr int N = S::N, NV = S::NV, NF = S::NF, EU = S::EU, EF = S::EF, EPB = S::EPB;
  constexpr int FQ = S::NFC * NF;
  __shared__ T su[EPB * EU];
  __shared__ int8_t need[EPB];
  if (d_M && *d_M < M) M = *d_M;  // the element count on the device (M is then a bound of it)
  const int64_t e0 = int64_t(blockIdx.x) * EPB;
  if (e0 >= M) return;
  const int ne = int((M - e0) < EPB ? (M - e0) : EPB);
  if (threadIdx.x < ne) need[threadIdx.x] = mask ? mask[e0 + threadIdx.x] : 1;
  __syncthreads();
  for (int k = threadIdx.x; k < ne * EU; k += blockDim.x)
    if (need[k / EU]) su[k] = Ar<T>::from_d(u[e0 * EU + k]);
  __syncthreads();
  for (int k = threadIdx.x; k < ne * FQ; k += blockDim.x) {
    const int le = k / FQ, r = k % FQ;
    if (!need[le]) continue;
    const int f = r / NF, q = r % NF;
    const T* lf = (f & 1) ? ops.lp : ops.lm;
    int pts[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) pts[j] = line_pt<DIM, NP>(f >> 1, q, j);
    T* to = tr + (e0 + le) * EF + f * NV * NF + q;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const T* ue = su + le * EU + v * N;
      T s = zero_t<T>();
#pragma unroll
      for (int j = 0; j < NP; ++j) s = fma_t(lf[j], ue[pts[j]], s);
      to[v * NF] = s;
    }
  }
}

// interface kernel: blocks [0, nb_hang) do hanging faces (one block slice per coarse face: Rusanov
// on every mortar piece, then the coarse side's L2 back-projection, owner-computes, Sec. 4.3), the
// others conforming faces (one thread per face point).  The heavier hanging blocks come first so
// that they are not left running alone at the end of the grid.
// block size of the interface kernel: 64 threads (more, smaller blocks spread one partial wave
// evenly over the SMs) unless one hanging face needs more threads than that
// faces per block (1..8, at most 512 threads) that leave the fewest idle lanes in whole warps
constexpr int face_fpb(int per) {
  int best = 1, bn = 0, bd = 1;
  for (int f = 1; f <= 8 && f * per <= 512; ++f) {
    const int n = f * per, d = (n + 31) / 32 * 32;
    if (n * bd > bn * d) {
      best = f;
      bn = n;
      bd = d;
    }
  }
  return best;
}

template <int DIM, int NP>
struct FaceCfg {
  static constexpr int PER = (1 << (DIM - 1)) * (DIM == 2 ? NP : NP * NP);  // threads per hanging face
  static constexpr int T0 = PER > 64 ? 128 : 64;
  static constexpr bool FULL = (T0 / PER) * PER * 10 >= T0 * 9;  // at most a tenth of T0 idle
  // otherwise (3D p = 2: one 36-point face per 64 threads) as many faces as fill whole warps
  static constexpr int FPB = FULL ? T0 / PER : face_fpb(PER);
  static constexpr int T = FULL ? T0 : (FPB * PER + 31) / 32 * 32;
};

template <int DIM, int NP, class T>
__global__ void __launch_bounds__(FaceCfg<DIM, NP>::T) k_faces_t(FaceArgs A, const __grid_constant__ OpsT<T> ops) {
  using S = Sz<DIM, NP>;
  constexpr int NV = S::NV, NF = S::NF, NFC = S::NFC, NSUB = S::NSUB;
  constexpr int PER = FaceCfg<DIM, NP>::PER, BT = FaceCfg<DIM, NP>::T;
  constexpr int FPB = FaceCfg<DIM, NP>::FPB;
  __shared__ T sF[FPB][NSUB][NV][NF];
  // 3D: the sum-factorised mortar stages' partial sums (interpolation HA, back-projection HB)
  constexpr int HA = 2 * NV * NP * NP, HB = NSUB * NV * NP * NP;
  __shared__ T sW[FPB][DIM == 3 ? (HA > HB ? HA : HB) : 1];
  const T* trace = static_cast<const T*>(A.trace);
  T* fcomm = static_cast<T*>(A.fcomm);
  const T gam = ops.gam, gm1 = ops.gm1, ngmh = ops.ngmh;
  const int tid = threadIdx.x;
  // the face lists and neighbour tables are fixed during a time step: they are read while the
  // element kernel this one depends on drains; the traces it wrote are read after the wait
  if (int64_t(blockIdx.x) >= A.nb_hang) {
    int64_t idx = (int64_t(blockIdx.x) - A.nb_hang) * BT + tid;
    int64_t face = idx / NF;
    int q = int(idx % NF);
    if (face >= A.n_conf) return;
    int32_t code = A.conf[face];
    int64_t e = code >> 2;
    int axis = code & 3;
    int64_t nb = A.nbr[e * NFC + 2 * axis + 1];
    pdl_wait_then_release();
    T qL[NV], qR[NV], F[NV];
    const T* tL = trace + ((e * NFC + 2 * axis + 1) * NV) * NF + q;
    const T* tR = trace + ((nb * NFC + 2 * axis) * NV) * NF + q;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      qL[v] = tL[v * NF];
      qR[v] = tR[v * NF];
    }
    rusanov2_t<DIM, T>(qL, qR, axis, gam, gm1, ngmh, F);
    T* fL = fcomm + ((e * NFC + 2 * axis + 1) * NV) * NF + q;
    T* fR = fcomm + ((nb * NFC + 2 * axis) * NV) * NF + q;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      fL[v * NF] = F[v];
      fR[v * NF] = F[v];
    }
    return;
  }
  const int64_t hb = int64_t(blockIdx.x);
  const int lf = tid / PER, r = tid % PER, s = r / NF, q = r % NF;
  const int64_t hf = hb * FPB + lf;
  const bool act = lf < FPB && hf < A.n_hang;
  int64_t ec = 0, ek = 0;
  int fc = 0;
  if (act) {
    const int32_t code = A.hang[hf];
    ec = code >> 3;
    fc = code & 7;
    ek = A.contrib[hf * 4 + s];
  }
  pdl_wait_then_release();
  const T* tc = trace + ((ec * NFC + fc) * NV) * NF;
  const int q0 = q % NP, h0 = s & 1;
  if (DIM == 3) {
    // the coarse trace's interpolation to the mortar pieces, sum-factorised across the face's
    // threads: first along the face's first axis for both halves, a1[h0][v][q0][j1], shared
    if (act)
      for (int k = r; k < HA; k += PER) {
        const int j1 = k % NP, qa = (k / NP) % NP, v = (k / (NP * NP)) % NV, ha = k / (NP * NP * NV);
        T a1 = zero_t<T>();
#pragma unroll
        for (int j0 = 0; j0 < NP; ++j0) a1 = fma_t(ops.I[ha][qa][j0], tc[v * NF + j0 + NP * j1], a1);
        sW[lf][k] = a1;
      }
    __syncthreads();
  }
  if (act) {
    int axis = fc >> 1, sidec = fc & 1;
    int fk = fc ^ 1;
    T uc[NV], uf[NV], F[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T acc = zero_t<T>();
      if (DIM == 2) {
#pragma unroll
        for (int j0 = 0; j0 < NP; ++j0) acc = fma_t(ops.I[h0][q0][j0], tc[v * NF + j0], acc);
      } else {
        // then along the second axis, per thread (the same operations in the same order as the
        // direct tensor-product sum)
        const int q1 = q / NP, h1 = s >> 1;
        const T* a1 = &sW[lf][((h0 * NV + v) * NP + q0) * NP];
#pragma unroll
        for (int j1 = 0; j1 < NP; ++j1) acc = fma_t(ops.I[h1][q1][j1], a1[j1], acc);
      }
      uc[v] = acc;
      uf[v] = trace[((ek * NFC + fk) * NV + v) * NF + q];
    }
    if (sidec)
      rusanov2_t<DIM, T>(uc, uf, axis, gam, gm1, ngmh, F);
    else
      rusanov2_t<DIM, T>(uf, uc, axis, gam, gm1, ngmh, F);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      fcomm[((ek * NFC + fk) * NV + v) * NF + q] = F[v];
      sF[lf][s][v][q] = F[v];
    }
  }
  __syncthreads();
  // back-projection onto the coarse face: its NV*NF outputs are spread over all PER threads of
  // the face (an idle lane costs the FP64 unit as much as a busy one); in 3D sum-factorised
  // across the threads, first along the first axis per mortar piece, b1[sp][v][q0][i1] (reusing
  // the interpolation's shared buffer), then each output along the second axis
  if (DIM == 3) {
    if (act)
      for (int k = r; k < HB; k += PER) {
        const int i1 = k % NP, qa = (k / NP) % NP, v = (k / (NP * NP)) % NV, sp = k / (NP * NP * NV);
        T b1 = zero_t<T>();
#pragma unroll
        for (int i0 = 0; i0 < NP; ++i0) b1 = fma_t(ops.P[sp & 1][qa][i0], sF[lf][sp][v][i0 + NP * i1], b1);
        sW[lf][k] = b1;
      }
    __syncthreads();
  }
  if (act) {
    for (int o = r; o < NV * NF; o += PER) {
      const int v = o / NF, qc = o % NF, qo = qc % NP;
      T acc = zero_t<T>();
#pragma unroll
      for (int sp = 0; sp < NSUB; ++sp) {
        if (DIM == 2) {
#pragma unroll
          for (int i0 = 0; i0 < NP; ++i0) acc = fma_t(ops.P[sp & 1][qo][i0], sF[lf][sp][v][i0], acc);
        } else {
          const int q1 = qc / NP, h1 = sp >> 1;
          const T* b1 = &sW[lf][((sp * NV + v) * NP + qo) * NP];
#pragma unroll
          for (int i1 = 0; i1 < NP; ++i1) acc = fma_t(ops.P[h1][q1][i1], b1[i1], acc);
        }
      }
      fcomm[((ec * NFC + fc) * NV + v) * NF + qc] = acc;
    }
  }
}

// Runge-Kutta combination type: FP64 for double and float (the mixed form keeps FP64 RK
// accumulation), double-word for ff.
template <class T>
struct RkT {
  using type = double;
};
template <>
struct RkT<ff> {
  using type = ff;
};

// Resident blocks the element kernel is compiled for: the FP32 form is bound by memory latency
// and wants every block shared memory allows (the register budget is set to fit them); the others
// keep the compiler's choice.
template <class T>
struct StageMinBlocks {
  static constexpr int value = std::is_same<T, float>::value ? 12 : 1;
};

// element stage: R = -sum_a (2/h) [ sum_j Dt_ij f_j + gL_i F(-1) + gR_i F(+1) ] along each axis
// (corrected-flux derivative of Sec. 2.1 with the correction folded into Dt; the interface kernel
// stores 2F and the slopes carry the 1/2), then out = a*un + b*us + c*R (Eq. rk3), and
// (optionally) the traces of out.  Phases: stage state -> pointwise fluxes -> volume sums
// sum_j Dt_ij f_j, all before the wait on the interface kernel; then its common fluxes ->
// correction terms, Runge-Kutta combination, traces.
template <int DIM, int NP, class T>
__global__ void __launch_bounds__(Sz<DIM, NP>::BT, StageMinBlocks<T>::value) k_stage_t(StageArgs A, const __grid_constant__ OpsT<T> ops) {
  using S = Sz<DIM, NP>;
  using RT = typename RkT<T>::type;
  constexpr int N = S::N, NV = S::NV, NF = S::NF, EU = S::EU, EF = S::EF;
  constexpr int EPB = S::EPB;
  __shared__ T su[EPB * EU];
  __shared__ T sfl[EPB * DIM * EU];
  __shared__ T sfc[EPB * EF];
  __shared__ double sh2[EPB];  // per element: c * (-2/h)
  __shared__ unsigned long long sg2[EPB];  // per element: the indicator's max |D rho|^2 (as bits)
  const T* fcomm = static_cast<const T*>(A.fcomm);
  T* trace_out = static_cast<T*>(A.trace_out);
  const int tid = threadIdx.x;
  const int64_t e0 = int64_t(blockIdx.x) * EPB;
  const int ne = int((A.M - e0) < EPB ? (A.M - e0) : EPB);
  // the stage's input state, the state at the start of the step and the keys come from earlier
  // launches than the interface kernel this one depends on, so they are read, and the pointwise
  // fluxes formed from them, while that kernel drains; the common fluxes are read after it.  Each
  // thread loads its own point; its u^n stays in registers for the Runge-Kutta combination.
  const int le = tid / N, i = tid % N;
  const bool act = le < ne;
  double unr[NV];
  if (act) {
    const int64_t b0 = (e0 + le) * EU + i;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      unr[v] = (A.rk & RK_A) ? A.un[b0 + v * N] : 0.0;
      su[le * EU + v * N + i] = Ar<T>::from_d(A.us[b0 + v * N]);
    }
  }
  // c * (-2/h): 2^depth * (2/L) is exact, so this equals the rounded -2^(depth+1)/L times c
  if (tid < ne) {
    sh2[tid] = -A.c * (double(1ull << A.g.depth(A.keys[e0 + tid])) * A.twoL);
    sg2[tid] = 0ull;
  }
  __syncthreads();
  const T gm1 = ops.gm1, ngmh = ops.ngmh;
  RT outv[NV];
  if (act) {
    const T* q = su + le * EU;
    T rho = q[i], rinv = rcp_t(rho), E = q[(NV - 1) * N + i];
    T vel[DIM];
    T m2 = zero_t<T>();
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      vel[b] = q[(1 + b) * N + i] * rinv;
      m2 = fma_t(q[(1 + b) * N + i], vel[b], m2);
    }
    T p = fma_t(ngmh, m2, gm1 * E);
    T Ep = E + p;
    // momentum flux m_b v_a, symmetric in (a, b): each off-diagonal product is formed once
    T mv[DIM][DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int b = a; b < DIM; ++b) {
        mv[a][b] = q[(1 + b) * N + i] * vel[a];
        mv[b][a] = mv[a][b];
      }
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      T* fa = sfl + (le * DIM + a) * EU;
      fa[i] = q[(1 + a) * N + i];
#pragma unroll
      for (int b = 0; b < DIM; ++b) fa[(1 + b) * N + i] = (a == b) ? mv[a][b] + p : mv[a][b];
      fa[(NV - 1) * N + i] = Ep * vel[a];
    }
  }
  __syncthreads();
  // volume part of the folded derivative, sum_a sum_j Dt_ij f_j, also before the wait: one FMA
  // chain per variable, the correction terms are added once the common fluxes are in
  T R[NV];
  if (act) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      int qf, ia;
      pt_split<DIM, NP>(i, a, &qf, &ia);
      const T* fa = sfl + (le * DIM + a) * EU;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T d = a == 0 ? ops.Dt[ia][0] * fa[v * N + line_pt<DIM, NP>(a, qf, 0)]
                     : fma_t(ops.Dt[ia][0], fa[v * N + line_pt<DIM, NP>(a, qf, 0)], R[v]);
#pragma unroll
        for (int j = 1; j < NP; ++j) d = fma_t(ops.Dt[ia][j], fa[v * N + line_pt<DIM, NP>(a, qf, j)], d);
        R[v] = d;
      }
    }
  }
  pdl_wait_then_release();
  for (int k = tid; k < ne * EF; k += blockDim.x) sfc[k] = fcomm[e0 * EF + k];
  __syncthreads();
  if (act) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      int qf, ia;
      pt_split<DIM, NP>(i, a, &qf, &ia);
      const T* Fm = sfc + le * EF + (2 * a) * NV * NF + qf;
      const T* Fp = sfc + le * EF + (2 * a + 1) * NV * NF + qf;
#pragma unroll
      for (int v = 0; v < NV; ++v) R[v] = fma_t(ops.gLh[ia], Fm[v * NF], fma_t(ops.gRh[ia], Fp[v * NF], R[v]));
    }
    const double cs = sh2[le];
    // u_s in FP64: the staged copy where it is exact (FP64 form), else the state in memory (an
    // L2 hit: this block read it at its start); kept out of registers to hold the occupancy
    double usr[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v)
      usr[v] = std::is_same<T, double>::value ? Ar<T>::to_d(su[le * EU + v * N + i])
                                              : A.us[(e0 + le) * EU + v * N + i];
    if constexpr (!std::is_same<T, ff>::value) {
      // FP64 combination (native FP64 and the mixed FP32 form).  The first stage (a = 0, b = 1)
      // is one FMA per value; the branch is uniform over the grid (kernel arguments), so the
      // other stages do not pay for it
      if (A.rk == RK_B1) {
#pragma unroll
        for (int v = 0; v < NV; ++v) outv[v] = fma(cs, Ar<T>::to_d(R[v]), usr[v]);
      } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          double o = fma(cs, Ar<T>::to_d(R[v]), (A.rk & RK_B1) ? usr[v] : A.b * usr[v]);
          if (A.rk & RK_A) o = fma(A.a, unr[v], o);
          outv[v] = o;
        }
      }
    } else {
      // double-word combination
      const ff bb = ff_from_double(A.b), cc = ff_from_double(cs), aa = ff_from_double(A.a);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        ff o = fma_t(bb, su[le * EU + v * N + i], cc * R[v]);
        if (A.rk & RK_A) o = fma_t(aa, ff_from_double(unr[v]), o);
        outv[v] = o;
      }
    }
  }
  __syncthreads();
  if (act) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      if constexpr (std::is_same<T, ff>::value)
        su[le * EU + v * N + i] = outv[v];
      else
        su[le * EU + v * N + i] = Ar<T>::from_d(outv[v]);
      A.out[(e0 + le) * EU + v * N + i] = Ar<RT>::to_d(outv[v]);
    }
  }
  __syncthreads();
  if constexpr (std::is_same<T, double>::value) {
    // the density-gradient indicator of the new state (FP64 form; the same arithmetic as the
    // indicator kernel): eta = 2 max_i |D_xi rho|, flags from the thresholds
    if (A.flags) {
      if (act) {
        const double* rho = su + le * EU;
        double g2 = 0.0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
          int qf, ia;
          pt_split<DIM, NP>(i, a, &qf, &ia);
          double d = 0.0;
#pragma unroll
          for (int j = 0; j < NP; ++j) d += ops.D[ia][j] * rho[line_pt<DIM, NP>(a, qf, j)];
          g2 += d * d;
        }
        atomicMax(&sg2[le], static_cast<unsigned long long>(__double_as_longlong(g2)));  // g2 >= 0
      }
      __syncthreads();
      if (act && i == 0) {
        const double val = 2.0 * sqrt(__longlong_as_double(static_cast<long long>(sg2[le])));
        A.flags[e0 + le] = int8_t(val > A.th_r ? 1 : (val < A.th_c ? -1 : 0));
      }
    }
  }
  if (trace_out) {
    // one thread per (element, face, face point), all variables from one set of indices
    constexpr int FQ = S::NFC * NF;
    for (int k = tid; k < ne * FQ; k += blockDim.x) {
      const int le2 = k / FQ, r = k % FQ;
      const int f = r / NF, qq = r % NF;
      const T* lf = (f & 1) ? ops.lp : ops.lm;
      int pts[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) pts[j] = line_pt<DIM, NP>(f >> 1, qq, j);
      T* to = trace_out + (e0 + le2) * EF + f * NV * NF + qq;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const T* ue = su + le2 * EU + v * N;
        if constexpr (std::is_same<T, ff>::value) {
          ffacc A{0.f, 0.f};
#pragma unroll
          for (int j = 0; j < NP; ++j) ffacc_fma(A, lf[j], ue[pts[j]]);
          to[v * NF] = ffacc_fin(A);
        } else {
          T s = zero_t<T>();
#pragma unroll
          for (int j = 0; j < NP; ++j) s = fma_t(lf[j], ue[pts[j]], s);
          to[v * NF] = s;
        }
      }
    }
  }
}

// ---- per-precision launch bodies (instantiated in fr_prec_*.cu) ----
#define FR_NP_DISPATCH(dim, p, ...)                                  \
  do {                                                               \
    int np_ = (p) + 1;                                               \
    if ((dim) == 2) {                                                \
      constexpr int DD = 2;                                          \
      if (np_ == 2) { constexpr int NN = 2; __VA_ARGS__; }           \
      else if (np_ == 3) { constexpr int NN = 3; __VA_ARGS__; }      \
      else if (np_ == 4) { constexpr int NN = 4; __VA_ARGS__; }      \
      else if (np_ == 5) { constexpr int NN = 5; __VA_ARGS__; }      \
      else return set_error(err, FR_EINVAL, "p out of range");     \
    } else if ((dim) == 3) {                                         \
      constexpr int DD = 3;                                          \
      if (np_ == 2) { constexpr int NN = 2; __VA_ARGS__; }           \
      else if (np_ == 3) { constexpr int NN = 3; __VA_ARGS__; }      \
      else if (np_ == 4) { constexpr int NN = 4; __VA_ARGS__; }      \
      else if (np_ == 5) { constexpr int NN = 5; __VA_ARGS__; }      \
      else return set_error(err, FR_EINVAL, "p out of range");     \
    } else {                                                         \
      return set_error(err, FR_EINVAL, "dim out of range");        \
    }                                                                \
  } while (0)

inline int ipow_k(int b, int e) {
  int r = 1;
  while (e-- > 0) r *= b;
  return r;
}

template <class T>
int launch_traces_impl(int dim, int p, const double* u, int64_t M, const DevOps& o, void* tr,
                       const int8_t* mask, cudaStream_t s, Err* err, const int64_t* d_M) {
  if (M <= 0) return 0;
  OpsT<T> ops = make_ops_t<T>(o);
  FR_NP_DISPATCH(dim, p, ({
                   using SS = Sz<DD, NN>;
                   const unsigned nb = unsigned((M + SS::EPB - 1) / SS::EPB);
                   launch_dependent(k_traces_t<DD, NN, T>, nb, SS::BT, s, u, M, ops, static_cast<T*>(tr), mask, d_M);
                 }));
  FR_LAUNCH_CHECK(err);
  return 0;
}

template <class T>
int launch_faces_impl(int dim, int p, FaceArgs A, const DevOps& o, cudaStream_t s, Err* err) {
  if (A.n_conf + A.n_hang == 0) return 0;
  OpsT<T> ops = make_ops_t<T>(o);
  set_gas(&ops, A.gamma);
  FR_NP_DISPATCH(dim, p, ({
                   using FC = FaceCfg<DD, NN>;
                   const int NF = DD == 2 ? NN : NN * NN;
                   A.nb_conf = (A.n_conf * NF + FC::T - 1) / FC::T;
                   A.nb_hang = (A.n_hang + FC::FPB - 1) / FC::FPB;
                   if (launch_dependent(k_faces_t<DD, NN, T>, unsigned(A.nb_conf + A.nb_hang), FC::T, s, A, ops) !=
                       cudaSuccess)
                     return set_error(err, FR_ECUDA, "interface kernel launch");
                 }));
  FR_LAUNCH_CHECK(err);
  return 0;
}

// Resident warps per SM allowed to the FP64 element kernel.  Its blocks are scheduled while the
// interface kernel they wait for still runs (dependent launch) and hold their slots while they
// wait; with the whole SM open to them (2D p = 3: 13 blocks of 4 warps, bounded by shared
// memory) they leave that kernel too few warps.  Measured on the 2D p = 3 workload: 8, 9, 10, 11
// and 16 resident blocks give +0.5, +0.7, +0.3, +0.15 and -1.4% against 13.  The other
// arithmetic forms keep the full residency.
constexpr int STAGE_F64_MAX_WARPS = 36;
template <int DIM, int NP, class T>
size_t stage_smem_pad() {
  static const size_t pad = std::is_same<T, double>::value
                                ? residency_pad(k_stage_t<DIM, NP, T>, Sz<DIM, NP>::BT, STAGE_F64_MAX_WARPS)
                                : 0;
  return pad;
}

template <class T>
int launch_stage_impl(int dim, int p, const StageArgs& A, const DevOps& o, cudaStream_t s, Err* err) {
  if (A.M <= 0) return 0;
  OpsT<T> ops = make_ops_t<T>(o);
  set_gas(&ops, A.gamma);
  FR_NP_DISPATCH(dim, p, ({
                   using SS = Sz<DD, NN>;
                   unsigned nb = unsigned((A.M + SS::EPB - 1) / SS::EPB);
                   if (launch_dependent_smem(k_stage_t<DD, NN, T>, nb, SS::BT, stage_smem_pad<DD, NN, T>(), s, A,
                                             ops) != cudaSuccess)
                     return set_error(err, FR_ECUDA, "element kernel launch");
                 }));
  FR_LAUNCH_CHECK(err);
  return 0;
}

}  // namespace frg
