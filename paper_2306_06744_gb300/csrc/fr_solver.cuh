// fr_solver.cuh -- launch interface of the FR kernels (fr_solver.cu).
#pragma once
#include "fr_internal.cuh"

namespace frg {

struct FaceArgs {
  const void* trace;      // [M][2dim][nv][Nf] traces of the current stage state (arithmetic type)
  void* fcomm;            // [M][2dim][nv][Nf] twice the common flux along +axis (arithmetic type)
  const int32_t* nbr;     // [M][2dim]
  const int32_t* conf;    // conforming faces: (minus element << 2) | axis
  const int32_t* hang;    // hanging faces: (coarse element << 3) | coarse face
  const int32_t* contrib; // [n_hang][4] fine elements in slot order
  int64_t n_conf, n_hang, nb_conf, nb_hang;
  double gamma;
};

struct StageArgs {
  const uint64_t* keys;
  const double* us;     // stage state
  const double* un;     // state at the start of the step (read only when a != 0)
  const void* fcomm;    // twice the common fluxes, in the arithmetic type
  double* out;          // a*un + b*us + c*R (may alias us or un element-wise)
  void* trace_out;      // traces of out in the arithmetic type, or null
  int64_t M;
  KG g;
  double twoL, gamma, a, b, c;  // twoL = 2 / L
  int rk;                       // RK_A: a != 0; RK_B1: b == 1 (integer tests, no FP64 compares per thread)
  int* status;                  // device word set by a tensor-core kernel whose completion wait gave up
  int8_t* flags;                // FP64 form: density-gradient flags of out (nullable)
  double th_r, th_c;            // their refine / coarsen thresholds
};

enum { RK_A = 1, RK_B1 = 2 };
inline int rk_mode(double a, double b) { return (a != 0.0 ? RK_A : 0) | (b == 1.0 ? RK_B1 : 0); }

struct Mesh;  // defined in fr_api.cu

int launch_exact(int dim, int p, const uint64_t* keys, int64_t M, const KG& g, double t,
                 const DevProblem& P, const DevOps& ops, double* u, cudaStream_t s, Err* err);
// prec: 0 FP64, 1 FP32 with FP64 Runge-Kutta combination, 2 TF32 and 3 bf16x3 tensor-core
// derivative (otherwise as 1; 3D p = 3), 4 double-word (two floats).  mask (nullable): traces only
// of the elements with a non-zero entry.  d_M (nullable): the element count on the device, M is then
// a bound of it
int launch_traces(int prec, int dim, int p, const double* u, int64_t M, const DevOps& ops, void* tr,
                  cudaStream_t s, Err* err, const int8_t* mask = nullptr, const int64_t* d_M = nullptr);
// bytes of one element's traces in the arithmetic type of `prec`
inline int trace_elem_bytes(int prec) { return (prec >= 1 && prec <= 3) ? 4 : 8; }
int launch_faces(int prec, int dim, int p, FaceArgs A, const DevOps& ops, cudaStream_t s, Err* err);
int launch_stage(int prec, int dim, int p, const StageArgs& A, const DevOps& ops, cudaStream_t s,
                 Err* err);
// per-precision instantiations (fr_prec_f64.cu, fr_prec_f32.cu, fr_prec_ff.cu)
#define FR_DECLARE_PREC(sfx)                                                                    \
  int launch_traces_##sfx(int dim, int p, const double* u, int64_t M, const DevOps& ops,        \
                          void* tr, const int8_t* mask, cudaStream_t s, Err* err,               \
                          const int64_t* d_M);                                                  \
  int launch_faces_##sfx(int dim, int p, FaceArgs A, const DevOps& ops, cudaStream_t s,         \
                         Err* err);                                                             \
  int launch_stage_##sfx(int dim, int p, const StageArgs& A, const DevOps& ops, cudaStream_t s, \
                         Err* err);
FR_DECLARE_PREC(f64)
FR_DECLARE_PREC(f32)
FR_DECLARE_PREC(ff)
// element stage of the tensor-core forms (fr_tc_stage.cu)
int launch_stage_tc(int prec, int dim, int p, const StageArgs& A, const DevOps& ops, cudaStream_t s, Err* err);
// indicator: mode 0 density gradient, 1 analytic centre; flags int8[M], eta double[M] (nullable)
int launch_indicator(int dim, int p, int mode, double th_r, double th_c, double t,
                     const uint64_t* keys, int64_t M, const KG& g, const DevProblem& P,
                     const DevOps& ops, const double* u, int8_t* flags, double* eta,
                     cudaStream_t s, Err* err);
// Traces carried over by the transfer (all null: none): an unchanged element's `bytes` of traces
// are copied from src (old elements) to dst (new elements); a refined or fused element's traces
// are computed from its new state (FP64 sums in the trace kernel's order) and stored in the
// arithmetic type `kind` of the traces (0 FP64, 1 FP32, 2 double-word).
struct TraceCopy {
  const void* src;
  void* dst;
  int kind;
  int bytes;
};
// the trace storage kind of a precision form (see TraceCopy)
inline int trace_kind(int prec) { return prec == 0 ? 0 : (prec == 4 ? 2 : 1); }
// d_M_new (nullable): device count of new leaves, M_new then an upper bound.  src/tag: the
// old->new mapping, or null: the kernel maps the new leaves itself (mapping failures set *bad)
int launch_transfer(int dim, int p, const KG& g, const uint64_t* old_keys, int64_t n_old, const uint64_t* new_keys,
                    const int32_t* src, const int8_t* tag, int32_t* bad, int64_t M_new, const int64_t* d_M_new,
                    const DevOps& ops, const double* u_old, double* u_new, const TraceCopy& tc, cudaStream_t s,
                    Err* err);
// norms: out[0] = sum w|J|(rho_ex-rho)^2, out[1..nv] integrals, out[nv+1] min rho, out[nv+2] min p
int launch_norms(int dim, int p, const uint64_t* keys, int64_t M, const KG& g, double t,
                 const DevProblem& P, const DevOps& ops, const double* u, double* d_partial,
                 int64_t nblocks_cap, double* d_out, cudaStream_t s, Err* err);
int norms_blocks(int dim, int p, int64_t M);
// largest |v|+c over all points, written to *d_max (as the bit pattern of a positive double)
int launch_maxspeed(int dim, int p, const double* u, int64_t M, double gamma,
                    unsigned long long* d_max, cudaStream_t s, Err* err);

}  // namespace frg
