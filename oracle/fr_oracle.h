/*
 * fr_oracle.h -- plain, slow, single-threaded CPU oracle for h-adaptive flux reconstruction
 * on Morton-ordered linear quadtrees/octrees (Wang, Witherden & Jameson, arXiv 2306.06744).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the GPU library against the paper.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may load it.  It
 * shares no code, header, table or constant generator with the GPU library; the two agree only
 * because both follow the paper.  Everything is FP64; loops are lexicographic and unfused.
 *
 * Layouts (canonical, shared by convention with the GPU library's C ABI, not by code):
 *   keys  : uint64 Morton IDs, [interleaved anchor bits][dim*(Dmax-D) zero pad][depth, m_b bits]
 *           (Sec. 2.2, Algorithm 1), sorted ascending (ancestors before descendants).
 *   u     : double[M][nv][N], N=(p+1)^dim, point index i = ix + n*iy + n*n*iz, x fastest.
 *   faces : f = 2*axis + side, side 0 = minus face, 1 = plus face; the matching face is f^1.
 *   conn  : per element and face: nbr (int32), ftype (0 conforming, 1 this element is the fine
 *           side of a hanging face, 2 this element is the coarse side), slot (int8: for ftype 1
 *           the contributor position on the coarse face, child bits of the in-face axes with the
 *           lower axis least significant, Sec. 3.3; 0 for ftype 2; -1 for conforming).  For
 *           ftype 2, nbr is the slot-0 contributor.
 *
 * Pins: every function is checked by the CPU test suite against facts that do not come from this
 * code (brute force on small trees, closed forms, invariants, textbook operators, the paper's
 * printed values).  Parity unpinned: the refine/coarsen thresholds of the density-gradient
 * indicator and the CFL time-step rule are choices of this build, not of the paper (the
 * indicator value eta itself is pinned).
 *
 * Return codes: 0 success, negative on error (message via oracle_last_error()).
 */
#ifndef FR_ORACLE_H
#define FR_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_EINVAL (-1)
#define ORACLE_EOVERFLOW (-3)

typedef struct {
  int32_t dim, p;          /* 2 or 3; polynomial degree 1..4                                */
  double L;                /* periodic domain [0,L]^dim                                     */
  int32_t Dbase, Dmax;     /* coarsest allowed depth and finest depth                       */
  double gamma;
  int32_t nvort;           /* number of vortices                                            */
  const double* vort;      /* [nvort][4]: xc, yc, beta (strength), core radius at t=0        */
  double uinf[3];          /* freestream velocity                                           */
  double rho_inf, p_inf;
  double cfl, dt;          /* dt > 0 fixes the step; else dt from the CFL rule               */
  int32_t adapt_every;
  int32_t indicator;       /* 0 density gradient, 1 analytic centre (Sec. 5.2), 2 external  */
  double th_refine, th_coarsen;
  int32_t precision;       /* ignored: the oracle is FP64                                    */
  int32_t init_passes;     /* <0: Dmax-Dbase passes of {IC, flag, adapt}                     */
} oracle_config;

typedef struct {
  double t, l2_rho;        /* time, L2 norm of the density error against the exact solution */
  double integral[5];      /* integral of each conserved variable over the domain            */
  double min_rho, min_p;
  int64_t M;
} oracle_norms_out;

typedef struct oracle_mesh oracle_mesh;

const char* oracle_last_error(void);

/* ---- primitives on host arrays ---- */
int oracle_morton_encode(int dim, int Dmax, int64_t n, const int32_t* boxes /*[n][4] depth,x,y,z*/,
                         uint64_t* keys);
int oracle_morton_decode(int dim, int Dmax, int64_t n, const uint64_t* keys, int32_t* boxes);
int oracle_linearise(int dim, int Dmax, const uint64_t* keys, int64_t n, uint64_t* out,
                     int64_t cap, int64_t* n_out);
/* Tree completion from points pts[n][dim] in [0,L)^dim: coarsest complete tree whose leaves are
   at depth >= Dmin and which holds every point's depth-Dmax cell as a leaf (Sec. 3.1). */
int oracle_tree_complete(int dim, int Dmin, int Dmax, double L, const double* pts, int64_t n,
                         uint64_t* out, int64_t cap, int64_t* n_out);
int oracle_balance(int dim, int Dmax, const uint64_t* keys, int64_t n, uint64_t* out, int64_t cap,
                   int64_t* n_out);
int oracle_adapt_keys(int dim, int Dbase, int Dmax, const uint64_t* keys, const int8_t* flags,
                      int64_t n, uint64_t* out, int64_t cap, int64_t* n_out);
int oracle_map(int dim, int Dmax, const uint64_t* old_keys, int64_t n_old, const uint64_t* new_keys,
               int64_t n_new, int32_t* src, int8_t* tag /* 0 copy, 1 refine, 2 coarsen */);
int oracle_conn(int dim, int Dmax, const uint64_t* keys, int64_t n, int32_t* nbr, int8_t* ftype,
                int8_t* slot);
/* 1D operators on Gauss-Legendre points: x[n], w[n], D[n][n] (D[i][j] = l_j'(x_i)),
   lm[n] = l_j(-1), lp[n] = l_j(+1), gL[n] = g_L'(x_i), gR[n] = g_R'(x_i). */
int oracle_operators(int p, double* x, double* w, double* D, double* lm, double* lp, double* gL,
                     double* gR);
/* value of the left correction function g_L(x) = right Radau polynomial of degree p+1 */
double oracle_correction_gL(int p, double x);
/* one SSP-RK3 step (Eq. rk3) of u' = lam*u, for pinning the Runge-Kutta combination */
double oracle_rk3_scalar(double lam, double u0, double dt);
/* transfer of one element: refine (child index c) or coarsen (children[2^dim][nv][N]) */
int oracle_prolong(int dim, int p, int nv, const double* parent, int child, double* out);
int oracle_restrict(int dim, int p, int nv, const double* children, double* out);
/* closed-form vortex state at physical points xyz[npts][3], time t */
int oracle_exact(const oracle_config* cfg, double t, int64_t npts, const double* xyz, double* q);

/* ---- mesh-level API: the same calls as the GPU library, prefixed ---- */
int oracle_mesh_init(const oracle_config* cfg, oracle_mesh** out);
void oracle_mesh_free(oracle_mesh* m);
int oracle_step(oracle_mesh* m, int nsteps);
int oracle_run(oracle_mesh* m, int nsteps); /* steps with adaptation every adapt_every steps */
int oracle_adapt(oracle_mesh* m, const int8_t* flags_or_null);
int oracle_flags(oracle_mesh* m, int8_t* flags, double* eta_or_null, int64_t cap);
int oracle_rhs(oracle_mesh* m, double* R, int64_t cap);
int oracle_norms(oracle_mesh* m, oracle_norms_out* out);
int oracle_get_leaves(oracle_mesh* m, uint64_t* keys, int64_t cap, int64_t* M);
int oracle_get_state(oracle_mesh* m, double* u, int64_t cap);
int oracle_set_state(oracle_mesh* m, const uint64_t* keys, int64_t M, const double* u);
int oracle_get_conn(oracle_mesh* m, int32_t* nbr, int8_t* ftype, int8_t* slot, int64_t cap);
int oracle_set_time(oracle_mesh* m, double t);
int oracle_get_info(oracle_mesh* m, double* t, double* dt, int64_t* M, int64_t* step);

#ifdef __cplusplus
}
#endif
#endif
