// fr_solver.cu -- flux reconstruction kernels for sm_103a (arXiv 2306.06744, Sec. 2.1 and 4.2-4.3):
// closed-form vortex state, face traces, interface fluxes (Rusanov on conforming faces, mortar
// projection at 2:1 hanging faces, owner-computes back-projection without atomics), the element
// stage (corrected-flux divergence folded with the DG correction, SSP-RK3 combination, traces of
// the new state), the adaptation indicator, solution transfer and deterministic norms.
// All arithmetic is FP64.  Kernels are instantiated per (dim, p+1) so every small contraction is
// fully unrolled.
#include <cmath>

#include "fr_internal.cuh"
#include "fr_kernels.cuh"
#include "fr_solver.cuh"

namespace frg {

// ---------------------------------------------------------------------------------------------
// Host: 1D operators on Gauss-Legendre points.  Nodes from their closed forms (n <= 5), weights as
// exact integrals of the Lagrange basis polynomials, barycentric Lagrange evaluation, and the DG
// correction derivatives from the lift identity g_L'(x_i) = -l_i(-1)/w_i, g_R'(x_i) = l_i(1)/w_i
// (Huynh's Radau correction recovers nodal DG, Sec. 2.1).
// ---------------------------------------------------------------------------------------------
namespace {

bool gl_nodes(int n, double* x) {
  switch (n) {
    case 2: {
      double a = 1.0 / std::sqrt(3.0);
      x[0] = -a; x[1] = a;
      return true;
    }
    case 3: {
      double a = std::sqrt(0.6);
      x[0] = -a; x[1] = 0.0; x[2] = a;
      return true;
    }
    case 4: {
      double r = 2.0 / 7.0 * std::sqrt(1.2);
      double a = std::sqrt(3.0 / 7.0 - r), b = std::sqrt(3.0 / 7.0 + r);
      x[0] = -b; x[1] = -a; x[2] = a; x[3] = b;
      return true;
    }
    case 5: {
      double r = 2.0 * std::sqrt(10.0 / 7.0);
      double a = std::sqrt(5.0 - r) / 3.0, b = std::sqrt(5.0 + r) / 3.0;
      x[0] = -b; x[1] = -a; x[2] = 0.0; x[3] = a; x[4] = b;
      return true;
    }
    default: return false;
  }
}

// barycentric weights lambda_j = 1 / prod_{k != j} (x_j - x_k)
void bary(int n, const double* x, double* lam) {
  for (int j = 0; j < n; ++j) {
    double pr = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) pr *= (x[j] - x[k]);
    lam[j] = 1.0 / pr;
  }
}

// l_j(t) for all j (second barycentric form; exact nodes handled explicitly)
void lag_all(int n, const double* x, const double* lam, double t, double* out) {
  for (int j = 0; j < n; ++j)
    if (t == x[j]) {
      for (int k = 0; k < n; ++k) out[k] = (k == j) ? 1.0 : 0.0;
      return;
    }
  double den = 0.0;
  for (int j = 0; j < n; ++j) den += lam[j] / (t - x[j]);
  for (int j = 0; j < n; ++j) out[j] = (lam[j] / (t - x[j])) / den;
}

// integral over [-1,1] of the j-th Lagrange polynomial, by expanding it in monomials
double lag_integral(int n, const double* x, int j) {
  double c[NPMAX + 1] = {1.0};  // coefficients of prod (t - x_k)/(x_j - x_k)
  int deg = 0;
  for (int k = 0; k < n; ++k) {
    if (k == j) continue;
    double s = 1.0 / (x[j] - x[k]);
    double nc[NPMAX + 1] = {0};
    for (int m = 0; m <= deg; ++m) {
      nc[m + 1] += c[m] * s;
      nc[m] -= c[m] * x[k] * s;
    }
    ++deg;
    for (int m = 0; m <= deg; ++m) c[m] = nc[m];
  }
  double I = 0.0;
  for (int m = 0; m <= deg; ++m)
    if (m % 2 == 0) I += 2.0 * c[m] / double(m + 1);
  return I;
}

}  // namespace

int build_ops(int p, DevOps* o) {
  int n = p + 1;
  *o = DevOps{};
  if (!gl_nodes(n, o->x)) return FR_EINVAL;
  double lam[NPMAX];
  bary(n, o->x, lam);
  for (int j = 0; j < n; ++j) o->w[j] = lag_integral(n, o->x, j);
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      o->D[i][j] = (lam[j] / lam[i]) / (o->x[i] - o->x[j]);
      s += o->D[i][j];
    }
    o->D[i][i] = -s;
  }
  lag_all(n, o->x, lam, -1.0, o->lm);
  lag_all(n, o->x, lam, 1.0, o->lp);
  for (int i = 0; i < n; ++i) {
    o->gL[i] = -o->lm[i] / o->w[i];
    o->gR[i] = o->lp[i] / o->w[i];
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) o->Dt[i][j] = o->D[i][j] - o->gL[i] * o->lm[j] - o->gR[i] * o->lp[j];
  for (int h = 0; h < 2; ++h)
    for (int i = 0; i < n; ++i) {
      double row[NPMAX];
      lag_all(n, o->x, lam, 0.5 * (o->x[i] + 2.0 * h - 1.0), row);
      for (int j = 0; j < n; ++j) o->I[h][i][j] = row[j];
    }
  for (int h = 0; h < 2; ++h)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) o->P[h][j][i] = 0.5 * (o->w[i] / o->w[j]) * o->I[h][i][j];
  return 0;
}

// ---------------------------------------------------------------------------------------------
// Device helpers and the remaining (FP64) kernels
// ---------------------------------------------------------------------------------------------
namespace {

// closed-form advected isentropic vortex (Sec. 5.2) at physical point X
__device__ void vortex_state(const DevProblem& P, int dim, double t, const double* X, double* q) {
  const double pi = 3.141592653589793238462643;
  double du = 0.0, dv = 0.0, dT = 0.0;
  for (int k = 0; k < P.nvort; ++k) {
    double xc = P.vort[k][0] + P.uinf[0] * t, yc = P.vort[k][1] + P.uinf[1] * t;
    double dx = X[0] - xc, dy = X[1] - yc;
    dx -= P.L * floor(dx / P.L + 0.5);
    dy -= P.L * floor(dy / P.L + 0.5);
    double beta = P.vort[k][2], R = P.vort[k][3];
    double r2 = (dx * dx + dy * dy) / (R * R);
    double ex = exp(0.5 * (1.0 - r2));
    du -= beta / (2.0 * pi) * (dy / R) * ex;
    dv += beta / (2.0 * pi) * (dx / R) * ex;
    dT -= (P.gamma - 1.0) * beta * beta / (8.0 * P.gamma * pi * pi) * exp(1.0 - r2);
  }
  double Tinf = P.p_inf / P.rho_inf;
  double T = Tinf + dT;
  double rho = P.rho_inf * pow(T / Tinf, 1.0 / (P.gamma - 1.0));
  double p = rho * T;
  double vel[3] = {P.uinf[0] + du, P.uinf[1] + dv, P.uinf[2]};
  double ke = 0.0;
  q[0] = rho;
  for (int b = 0; b < dim; ++b) {
    q[1 + b] = rho * vel[b];
    ke += 0.5 * rho * vel[b] * vel[b];
  }
  q[1 + dim] = p / (P.gamma - 1.0) + ke;
}

template <int DIM, int NP>
__device__ __forceinline__ void point_xyz(const KG& g, double L, uint64_t key, int i,
                                          const DevOps& ops, double* X, double* h_out) {
  uint32_t a[3] = {0, 0, 0};
  deinterleave<DIM>(g.raw(key), a);
  int d = g.depth(key);
  double fine = L / double(1ull << g.Dmax);
  double h = L / double(1ull << d);
  int ii[3] = {i % NP, (i / NP) % NP, DIM == 3 ? i / (NP * NP) : 0};
  X[2] = 0.0;
#pragma unroll
  for (int b = 0; b < DIM; ++b) X[b] = double(a[b]) * fine + 0.5 * h * (ops.x[ii[b]] + 1.0);
  *h_out = h;
}

// ---------------------------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------------------------
template <int DIM, int NP>
__global__ void k_exact(const uint64_t* __restrict__ keys, int64_t M, KG g, double t,
                        const __grid_constant__ DevProblem P, const __grid_constant__ DevOps ops,
                        double* __restrict__ u) {
  using S = Sz<DIM, NP>;
  int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= M * S::N) return;
  int64_t e = idx / S::N;
  int i = int(idx % S::N);
  double X[3], h, q[5];
  point_xyz<DIM, NP>(g, P.L, keys[e], i, ops, X, &h);
  vortex_state(P, DIM, t, X, q);
#pragma unroll
  for (int v = 0; v < S::NV; ++v) u[(e * S::NV + v) * S::N + i] = q[v];
}

// traces tr[e][f][v][q] = sum_j l_j(+-1) u[e][v][line point j]  (mortar procedure step 1)
// Adaptation indicator, one thread per element.  Mode 0 (density gradient, a choice of this
// library): eta = h max_i |grad rho(x_i)| with the uncorrected local derivative (2/h) D rho, so
// eta = 2 max_i |D_xi rho|.  Mode 1 (analytic centre, Sec. 5.2): compare the numbers of points
// closer than th_r and farther than th_c from the nearest vortex axis.
template <int DIM, int NP>
__global__ void k_indicator(const uint64_t* __restrict__ keys, int64_t M, KG g, int mode,
                            double th_r, double th_c, double t, const __grid_constant__ DevProblem P,
                            const __grid_constant__ DevOps ops, const double* __restrict__ u,
                            int8_t* __restrict__ flags, double* __restrict__ eta) {
  pdl_wait_then_release();
  using S = Sz<DIM, NP>;
  int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= M) return;
  const double* rho = u + e * S::EU;
  int8_t f = 0;
  double val = 0.0;
  if (mode == 0) {
    double gmax = 0.0;
    for (int i = 0; i < S::N; ++i) {
      double g2 = 0.0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        int qf, ia;
        pt_split<DIM, NP>(i, a, &qf, &ia);
        double d = 0.0;
#pragma unroll
        for (int j = 0; j < NP; ++j) d += ops.D[ia][j] * __ldg(rho + line_pt<DIM, NP>(a, qf, j));
        g2 += d * d;
      }
      gmax = fmax(gmax, g2);
    }
    val = 2.0 * sqrt(gmax);
    f = val > th_r ? 1 : (val < th_c ? -1 : 0);
  } else {
    int nin = 0, nout = 0;
    uint64_t key = keys[e];
    for (int i = 0; i < S::N; ++i) {
      double X[3], h;
      point_xyz<DIM, NP>(g, P.L, key, i, ops, X, &h);
      double rmin = 1e300;
      for (int k = 0; k < P.nvort; ++k) {
        double dx = X[0] - (P.vort[k][0] + P.uinf[0] * t), dy = X[1] - (P.vort[k][1] + P.uinf[1] * t);
        dx -= P.L * floor(dx / P.L + 0.5);
        dy -= P.L * floor(dy / P.L + 0.5);
        rmin = fmin(rmin, sqrt(dx * dx + dy * dy));
      }
      nin += rmin < th_r;
      nout += rmin > th_c;
    }
    val = double(nin - nout);
    f = nin > nout ? 1 : (nin < nout ? -1 : 0);
  }
  flags[e] = f;
  if (eta) eta[e] = val;
}

// Solution transfer (Sec. 4.2): copy; interpolation of the old (ancestor) polynomial at the new
// points; L2 projection of 2^dim fused children onto the parent.  Both non-trivial cases are
// tensor products of 1D operators and are applied axis by axis (sum factorisation: DIM
// contractions of length n per output value instead of one of length N): for refinement the
// 1D Lagrange weights of the ancestor at the new points, for fusion the 1D projection operators
// P (exact-quadrature mass and cross-mass matrices), one child after the other.
// Blocks of EPB whole elements, one thread per point (as the element kernel).  Without a mapping
// (src null) each element's first thread maps its new leaf (one lower bound) into shared memory,
// so the adaptation needs no separate mapping kernel.
template <int DIM, int NP>
__global__ void __launch_bounds__(Sz<DIM, NP>::BT) k_transfer(KG g, const uint64_t* __restrict__ old_keys,
                                                              int64_t n_old, const uint64_t* __restrict__ new_keys,
                                                              const int32_t* __restrict__ src,
                                                              const int8_t* __restrict__ tag, int32_t* bad,
                                                              int64_t Mn_ub, const int64_t* __restrict__ d_Mn,
                                                              const __grid_constant__ DevOps ops,
                                                              const double* __restrict__ uo,
                                                              double* __restrict__ un, const TraceCopy tc) {
  pdl_wait_then_release();
  using S = Sz<DIM, NP>;
  constexpr int N = S::N, NV = S::NV, EU = S::EU, EPB = S::EPB;
  __shared__ double sa[EPB][EU], sb[EPB][EU];
  __shared__ double sw[EPB][DIM][NP][NP];  // refinement: 1D weights w[a][i][m] = l_m(xi_a(i))
  __shared__ int32_t s_src[EPB];
  __shared__ int8_t s_tag[EPB];
  __shared__ int s_rounds;
  const int64_t Mn = (d_Mn && *d_Mn < Mn_ub) ? *d_Mn : Mn_ub;
  const int64_t j0 = int64_t(blockIdx.x) * EPB;
  const int le = threadIdx.x / N, i = threadIdx.x % N;
  const int64_t j = j0 + le;
  const bool act = le < EPB && j < Mn;
  if (threadIdx.x == 0) s_rounds = 0;
  if (act && i == 0) {
    if (src) {
      s_src[le] = src[j];
      s_tag[le] = tag[j];
    } else {
      map_leaf<DIM>(old_keys, n_old, new_keys[j], g, &s_src[le], &s_tag[le], bad);
    }
  }
  __syncthreads();
  const int64_t sidx = act ? s_src[le] : 0;
  const int tg = act ? s_tag[le] : 0;
  const int ii[3] = {i % NP, (i / NP) % NP, DIM == 3 ? i / (NP * NP) : 0};
  if (act && tg == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) un[(j * NV + v) * N + i] = uo[(sidx * NV + v) * N + i];
    // an unchanged element keeps its traces: copied as 8-byte words
    if (tc.dst) {
      const int w = tc.bytes >> 3;
      const uint64_t* a = static_cast<const uint64_t*>(tc.src) + sidx * w;
      uint64_t* b = static_cast<uint64_t*>(tc.dst) + j * w;
      for (int k = i; k < w; k += N) b[k] = a[k];
    }
  }
  // rounds of the contraction: 1 for a refined element, 2^dim (one per child) for a fused one
  if (act && i == 0 && tg != 0) atomicMax(&s_rounds, tg == 1 ? 1 : (1 << DIM));
  if (act && tg == 1) {
    // 1D Lagrange weights of the ancestor at the new element's points along each axis
    const uint64_t kA = old_keys[sidx], kK = new_keys[j];
    uint32_t xa[3] = {0, 0, 0}, xk[3] = {0, 0, 0};
    deinterleave<DIM>(g.raw(kA), xa);
    deinterleave<DIM>(g.raw(kK), xk);
    const double wA = double(g.width(g.depth(kA))), wK = double(g.width(g.depth(kK)));
    for (int w = i; w < DIM * NP * NP; w += N) {
      const int a = w / (NP * NP), ia = (w / NP) % NP, m = w % NP;
      const double xi = -1.0 + 2.0 * (double(xk[a] - xa[a]) + 0.5 * (ops.x[ia] + 1.0) * wK) / wA;
      double pr = 1.0;
#pragma unroll
      for (int k = 0; k < NP; ++k)
        if (k != m) pr *= (xi - ops.x[k]) / (ops.x[m] - ops.x[k]);
      sw[le][a][ia][m] = pr;
    }
  }
  __syncthreads();
  const int rounds = s_rounds;
  double acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.0;
  const bool work = act && tg != 0;
  for (int r = 0; r < rounds; ++r) {
    // the round's source: the ancestor (refinement) or child r (fusion)
    const bool live = work && (tg == 2 || r == 0);
    if (live) {
      const int64_t se = tg == 2 ? sidx + r : sidx;
#pragma unroll
      for (int v = 0; v < NV; ++v) sa[le][v * N + i] = uo[(se * NV + v) * N + i];
    }
    __syncthreads();
    // axis by axis: along x from sa into sb, along y from sb into sa, along z from sa into sb
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      double* in = (a & 1) ? sb[le] : sa[le];
      double* out = (a & 1) ? sa[le] : sb[le];
      if (live) {
        const int h = (r >> a) & 1;
        const int stride = a == 0 ? 1 : (a == 1 ? NP : NP * NP);
        const int base = i - ii[a] * stride;  // the point with index 0 along axis a
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          double t = 0.0;
#pragma unroll
          for (int m = 0; m < NP; ++m) {
            const double wgt = tg == 1 ? sw[le][a][ii[a]][m] : ops.P[h][ii[a]][m];
            t = fma(wgt, in[v * N + base + m * stride], t);
          }
          if (a == DIM - 1)
            acc[v] += t;
          else
            out[v * N + i] = t;
        }
      }
      if (a < DIM - 1) __syncthreads();
    }
    __syncthreads();  // the next round overwrites sa
  }
  if (work) {
#pragma unroll
    for (int v = 0; v < NV; ++v) un[(j * NV + v) * N + i] = acc[v];
  }
  if (tc.dst && rounds > 0) {
    // the traces of this block's refined and fused elements, from their new state staged in
    // shared memory (the last round ended with a barrier): one thread per (element, face, face
    // point), all variables, the same sums in the same order as the trace kernel in FP64
    constexpr int NF = S::NF, FQ = S::NFC * NF, EF = S::EF;
    if (work) {
#pragma unroll
      for (int v = 0; v < NV; ++v) sa[le][v * N + i] = acc[v];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < EPB * FQ; k += blockDim.x) {
      const int le2 = k / FQ, r = k % FQ;
      if (j0 + le2 >= Mn || s_tag[le2] == 0) continue;
      const int f = r / NF, q = r % NF;
      const double* lf = (f & 1) ? ops.lp : ops.lm;
      const int64_t o = (j0 + le2) * EF + f * NV * NF + q;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        double t = 0.0;
#pragma unroll
        for (int m = 0; m < NP; ++m) t = fma(lf[m], sa[le2][v * N + line_pt<DIM, NP>(f >> 1, q, m)], t);
        if (tc.kind == 0)
          static_cast<double*>(tc.dst)[o + v * NF] = t;
        else if (tc.kind == 1)
          static_cast<float*>(tc.dst)[o + v * NF] = __double2float_rn(t);
        else
          static_cast<ff*>(tc.dst)[o + v * NF] = ff_from_double(t);
      }
    }
  }
}

// Norms: per-element sums, block tree reduction in fixed order, then one block over the partials.
constexpr int NRM_T = 128, NRM_W = 8;
template <int DIM, int NP>
__global__ void __launch_bounds__(NRM_T) k_norms(const uint64_t* __restrict__ keys, int64_t M, KG g,
                                                 double t, const __grid_constant__ DevProblem P,
                                                 const __grid_constant__ DevOps ops,
                                                 const double* __restrict__ u,
                                                 double* __restrict__ partial) {
  using S = Sz<DIM, NP>;
  __shared__ double sm[NRM_W][NRM_T];
  int64_t e = int64_t(blockIdx.x) * NRM_T + threadIdx.x;
  double acc[NRM_W];
  for (int k = 0; k < NRM_W; ++k) acc[k] = 0.0;
  acc[S::NV + 1] = 1e300;
  acc[S::NV + 2] = 1e300;
  if (e < M) {
    uint64_t key = keys[e];
    for (int i = 0; i < S::N; ++i) {
      double X[3], h, qe[5], q[5];
      point_xyz<DIM, NP>(g, P.L, key, i, ops, X, &h);
      vortex_state(P, DIM, t, X, qe);
      double Wt = ops.w[i % NP] * ops.w[(i / NP) % NP];
      if (DIM == 3) Wt *= ops.w[i / (NP * NP)];
      double J = 0.5 * h * 0.5 * h;
      if (DIM == 3) J *= 0.5 * h;
#pragma unroll
      for (int v = 0; v < S::NV; ++v) q[v] = u[(e * S::NV + v) * S::N + i];
      double d = qe[0] - q[0];
      acc[0] += Wt * J * d * d;
#pragma unroll
      for (int v = 0; v < S::NV; ++v) acc[1 + v] += Wt * J * q[v];
      double m2 = 0.0;
#pragma unroll
      for (int b = 0; b < DIM; ++b) m2 += q[1 + b] * q[1 + b];
      double p = (P.gamma - 1.0) * (q[S::NV - 1] - 0.5 * m2 / q[0]);
      acc[S::NV + 1] = fmin(acc[S::NV + 1], q[0]);
      acc[S::NV + 2] = fmin(acc[S::NV + 2], p);
    }
  }
  for (int k = 0; k < NRM_W; ++k) sm[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int st = NRM_T / 2; st > 0; st >>= 1) {
    if (int(threadIdx.x) < st)
      for (int k = 0; k < NRM_W; ++k) {
        double a = sm[k][threadIdx.x], b = sm[k][threadIdx.x + st];
        sm[k][threadIdx.x] = (k == S::NV + 1 || k == S::NV + 2) ? fmin(a, b) : a + b;
      }
    __syncthreads();
  }
  if (threadIdx.x < NRM_W) partial[int64_t(blockIdx.x) * NRM_W + threadIdx.x] = sm[threadIdx.x][0];
}

__global__ void __launch_bounds__(NRM_T) k_norms_final(const double* __restrict__ partial,
                                                       int64_t nb, int nv, double* __restrict__ out) {
  __shared__ double sm[NRM_W][NRM_T];
  double acc[NRM_W];
  for (int k = 0; k < NRM_W; ++k) acc[k] = (k == nv + 1 || k == nv + 2) ? 1e300 : 0.0;
  for (int64_t b = threadIdx.x; b < nb; b += NRM_T)
    for (int k = 0; k < NRM_W; ++k) {
      double x = partial[b * NRM_W + k];
      acc[k] = (k == nv + 1 || k == nv + 2) ? fmin(acc[k], x) : acc[k] + x;
    }
  for (int k = 0; k < NRM_W; ++k) sm[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int st = NRM_T / 2; st > 0; st >>= 1) {
    if (int(threadIdx.x) < st)
      for (int k = 0; k < NRM_W; ++k) {
        double a = sm[k][threadIdx.x], b = sm[k][threadIdx.x + st];
        sm[k][threadIdx.x] = (k == nv + 1 || k == nv + 2) ? fmin(a, b) : a + b;
      }
    __syncthreads();
  }
  if (threadIdx.x < NRM_W) out[threadIdx.x] = sm[threadIdx.x][0];
}

template <int DIM, int NP>
__global__ void k_maxspeed(const double* __restrict__ u, int64_t M, double gam,
                           unsigned long long* dmax) {
  using S = Sz<DIM, NP>;
  int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= M * S::N) return;
  int64_t e = idx / S::N;
  int i = int(idx % S::N);
  const double* q = u + e * S::EU + i;
  double rho = q[0], m2 = 0.0;
#pragma unroll
  for (int b = 0; b < DIM; ++b) m2 += q[(1 + b) * S::N] * q[(1 + b) * S::N];
  double p = (gam - 1.0) * (q[(S::NV - 1) * S::N] - 0.5 * m2 / rho);
  double s = sqrt(m2) / rho + sqrt(gam * p / rho);
  if (s > 0.0) atomicMax(dmax, (unsigned long long)__double_as_longlong(s));
}

inline unsigned nb_of(int64_t n, int b) { return unsigned((n + b - 1) / b); }

}  // namespace

// ---------------------------------------------------------------------------------------------
// Launchers: dispatch on (dim, p+1)
// ---------------------------------------------------------------------------------------------
#define FR_DISPATCH(dim, p, ...)                                        \
  do {                                                                  \
    int np_ = (p) + 1;                                                  \
    if ((dim) == 2) {                                                   \
      constexpr int DD = 2;                                             \
      if (np_ == 2) { constexpr int NN = 2; __VA_ARGS__; }              \
      else if (np_ == 3) { constexpr int NN = 3; __VA_ARGS__; }         \
      else if (np_ == 4) { constexpr int NN = 4; __VA_ARGS__; }         \
      else if (np_ == 5) { constexpr int NN = 5; __VA_ARGS__; }         \
      else return set_error(err, FR_EINVAL, "p out of range");        \
    } else if ((dim) == 3) {                                            \
      constexpr int DD = 3;                                             \
      if (np_ == 2) { constexpr int NN = 2; __VA_ARGS__; }              \
      else if (np_ == 3) { constexpr int NN = 3; __VA_ARGS__; }         \
      else if (np_ == 4) { constexpr int NN = 4; __VA_ARGS__; }         \
      else if (np_ == 5) { constexpr int NN = 5; __VA_ARGS__; }         \
      else return set_error(err, FR_EINVAL, "p out of range");        \
    } else {                                                            \
      return set_error(err, FR_EINVAL, "dim out of range");           \
    }                                                                   \
  } while (0)

static int ipow(int b, int e) {
  int r = 1;
  while (e-- > 0) r *= b;
  return r;
}

int launch_exact(int dim, int p, const uint64_t* keys, int64_t M, const KG& g, double t,
                 const DevProblem& P, const DevOps& ops, double* u, cudaStream_t s, Err* err) {
  if (M <= 0) return 0;
  int64_t T = M * ipow(p + 1, dim);
  FR_DISPATCH(dim, p, (k_exact<DD, NN><<<nb_of(T, 128), 128, 0, s>>>(keys, M, g, t, P, ops, u)));
  FR_LAUNCH_CHECK(err);
  return 0;
}

int launch_traces(int prec, int dim, int p, const double* u, int64_t M, const DevOps& ops, void* tr,
                  cudaStream_t s, Err* err, const int8_t* mask, const int64_t* d_M) {
  if (prec >= 1 && prec <= 3) return launch_traces_f32(dim, p, u, M, ops, tr, mask, s, err, d_M);
  if (prec == 4) return launch_traces_ff(dim, p, u, M, ops, tr, mask, s, err, d_M);
  return launch_traces_f64(dim, p, u, M, ops, tr, mask, s, err, d_M);
}

int launch_faces(int prec, int dim, int p, FaceArgs A, const DevOps& ops, cudaStream_t s, Err* err) {
  if (prec >= 1 && prec <= 3) return launch_faces_f32(dim, p, A, ops, s, err);
  if (prec == 4) return launch_faces_ff(dim, p, A, ops, s, err);
  return launch_faces_f64(dim, p, A, ops, s, err);
}

int launch_stage(int prec, int dim, int p, const StageArgs& A, const DevOps& ops, cudaStream_t s,
                 Err* err) {
  if (prec == 1) return launch_stage_f32(dim, p, A, ops, s, err);
  if (prec == 2 || prec == 3) return launch_stage_tc(prec, dim, p, A, ops, s, err);
  if (prec == 4) return launch_stage_ff(dim, p, A, ops, s, err);
  return launch_stage_f64(dim, p, A, ops, s, err);
}

int launch_indicator(int dim, int p, int mode, double th_r, double th_c, double t,
                     const uint64_t* keys, int64_t M, const KG& g, const DevProblem& P,
                     const DevOps& ops, const double* u, int8_t* flags, double* eta,
                     cudaStream_t s, Err* err) {
  if (M <= 0) return 0;
  FR_DISPATCH(dim, p, (launch_dependent(k_indicator<DD, NN>, nb_of(M, 128), 128, s, keys, M, g, mode, th_r, th_c, t, P,
                                        ops, u, flags, eta)));
  FR_LAUNCH_CHECK(err);
  return 0;
}

int launch_transfer(int dim, int p, const KG& g, const uint64_t* old_keys, int64_t n_old, const uint64_t* new_keys,
                    const int32_t* src, const int8_t* tag, int32_t* bad, int64_t M_new, const int64_t* d_M_new,
                    const DevOps& ops, const double* u_old, double* u_new, const TraceCopy& tc, cudaStream_t s,
                    Err* err) {
  if (M_new <= 0) return 0;
  FR_DISPATCH(dim, p, ({
                using SS = Sz<DD, NN>;
                launch_dependent(k_transfer<DD, NN>, unsigned((M_new + SS::EPB - 1) / SS::EPB), SS::BT, s, g,
                                 old_keys, n_old, new_keys, src, tag, bad, M_new, d_M_new, ops, u_old, u_new, tc);
              }));
  FR_LAUNCH_CHECK(err);
  return 0;
}

int norms_blocks(int dim, int p, int64_t M) {
  (void)dim;
  (void)p;
  return int((M + NRM_T - 1) / NRM_T);
}

int launch_norms(int dim, int p, const uint64_t* keys, int64_t M, const KG& g, double t,
                 const DevProblem& P, const DevOps& ops, const double* u, double* d_partial,
                 int64_t nblocks_cap, double* d_out, cudaStream_t s, Err* err) {
  int64_t nb = (M + NRM_T - 1) / NRM_T;
  if (nb > nblocks_cap) return set_error(err, FR_EINVAL, "norms scratch too small");
  if (nb > 0) {
    FR_DISPATCH(dim, p, (k_norms<DD, NN><<<unsigned(nb), NRM_T, 0, s>>>(keys, M, g, t, P, ops, u, d_partial)));
    FR_LAUNCH_CHECK(err);
  }
  k_norms_final<<<1, NRM_T, 0, s>>>(d_partial, nb, dim + 2, d_out);
  FR_LAUNCH_CHECK(err);
  return 0;
}

int launch_maxspeed(int dim, int p, const double* u, int64_t M, double gamma,
                    unsigned long long* d_max, cudaStream_t s, Err* err) {
  FR_CUDA(err, cudaMemsetAsync(d_max, 0, sizeof(unsigned long long), s));
  if (M <= 0) return 0;
  int64_t T = M * ipow(p + 1, dim);
  FR_DISPATCH(dim, p, (k_maxspeed<DD, NN><<<nb_of(T, 128), 128, 0, s>>>(u, M, gamma, d_max)));
  FR_LAUNCH_CHECK(err);
  return 0;
}

}  // namespace frg
