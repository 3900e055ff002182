// fr_api.cu -- the C ABI of include/fr.h: mesh object, time stepping, adaptation orchestration
// (flags -> edit -> 2:1 balance -> mapping -> transfer -> connectivity), face lists, host I/O and
// the device-array tree primitives.
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>

#include "fr_internal.cuh"
#include "fr_mlp.cuh"
#include "fr_solver.cuh"

using namespace frg;

struct fr_mesh {
  Err err;
  fr_config cfg{};
  std::vector<double> vort;
  int dim = 2, p = 1, n = 2, N = 4, Nf = 2, nv = 4, nfc = 4, EU = 16, EF = 32;
  KG g{};
  DevOps ops{};
  DevProblem prob{};
  cudaStream_t stream = nullptr;
  fr_allocator user{};
  bool has_user = false;
  BlockCache cache;
  Alloc A;
  double t = 0.0, dt = 0.0;
  int64_t step = 0, M = 0;
  Buf<uint64_t> keys;
  Buf<double> u, w, trace, fcomm;
  Buf<int32_t> nbr, conf, hang, contrib;
  Buf<int8_t> ftype, slot, flags;
  int64_t n_conf = 0, n_hang = 0;
  bool traces_ok = false;  // trace holds the traces of the current state u
  bool flags_fresh = false;  // flags hold the density-gradient flags of u (from the last stage)
  Buf<double> norm_part, norm_out;
  Buf<unsigned long long> dmax;
  Buf<float> mlp_params;  // learned indicator weights (FP32 master copy), empty if none
  // device words read back together at the end of an adaptation: the adaptation's control block
  // (CTL_SLOTS), its two error flags, and the status word a tensor-core kernel sets when its
  // completion wait gave up
  Buf<int64_t> ctlblk;
  int32_t* status = nullptr;
  // pinned host words mapped for the device: the adaptation's connectivity kernel publishes the
  // ctlblk words there followed by a sequence number (null: read back by copy and synchronise)
  int64_t* pub_h = nullptr;
  int64_t* pub_d = nullptr;
  int64_t pub_seq = 0;
  int64_t mlp_n = 0;
  // measurement: event pairs around interface (kind 0) and element (kind 1) launches
  struct Rec {
    int kind;
    cudaEvent_t a, b;
    int64_t points;
  };
  bool prof = false;
  int prof_stride = 1;     // time every prof_stride-th stage (interface + element kernel)
  int64_t prof_count = 0;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<Rec> recs;
  int64_t launches0 = 0;
  cudaEvent_t next_event() {
    if (ev_used == ev_pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      ev_pool.push_back(e);
    }
    return ev_pool[ev_used++];
  }
};

namespace {

constexpr int TB = 256;
// the mesh's block of device words (fr_mesh::ctlblk): control block, error flags, status word
constexpr int CTLBLK_BAD = CTL_SLOTS, CTLBLK_STATUS = CTL_SLOTS + 1, CTLBLK_WORDS = CTL_SLOTS + 2;
inline unsigned nblk(int64_t n, int b = TB) { return unsigned((n + b - 1) / b); }

template <int DIM>
__global__ void k_face_write(const int8_t* __restrict__ ftype, const int32_t* __restrict__ contrib,
                             int64_t M_ub, const int64_t* __restrict__ d_M, const Offs O,
                             int32_t* __restrict__ conf, int32_t* __restrict__ hang, int32_t* __restrict__ hcon) {
  pdl_wait_then_release();
  int64_t grand;
  const int64_t base = offs_base(O, int64_t(blockIdx.x) * blockDim.x, &grand);
  int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= M_ub || (d_M && e >= *d_M)) return;
  const int64_t off = O.offs[e] + base;  // packed: conforming count low, hanging count high
  int64_t a = off & 0xFFFFFFFFll, b = off >> 32;
#pragma unroll
  for (int f = 0; f < 2 * DIM; ++f) {
    int8_t t = ftype[e * 2 * DIM + f];
    if ((f & 1) && t == 0) conf[a++] = int32_t((e << 2) | (f >> 1));
    if (t == 2) {
      hang[b] = int32_t((e << 3) | f);
      for (int s = 0; s < 4; ++s) hcon[b * 4 + s] = contrib[(e * 2 * DIM + f) * 4 + s];
      ++b;
    }
  }
}

int check_cfg(const fr_config* c, Err* err) {
  if (!c) return set_error(err, FR_EINVAL, "null config");
  if (c->dim != 2 && c->dim != 3) return set_error(err, FR_EINVAL, "dim must be 2 or 3");
  if (c->p < 1 || c->p > 4) return set_error(err, FR_EINVAL, "p must be in 1..4");
  if (c->Dmax < 1 || c->Dmax > 30) return set_error(err, FR_EINVAL, "Dmax out of range");
  if (c->dim * c->Dmax + depth_bits(c->Dmax) > 63)
    return set_error(err, FR_EINVAL, "dim*Dmax + depth bits exceeds 63");
  if (c->dim == 3 && c->Dmax > 19) return set_error(err, FR_EINVAL, "Dmax > 19 in 3D");
  if (c->Dbase < 1 || c->Dbase > c->Dmax) return set_error(err, FR_EINVAL, "Dbase out of range");
  if (int64_t(1) << (c->dim * c->Dbase) > (int64_t(1) << 30))
    return set_error(err, FR_EINVAL, "base level too large");
  if (!(c->L > 0) || !(c->gamma > 1.0) || !(c->rho_inf > 0) || !(c->p_inf > 0))
    return set_error(err, FR_EINVAL, "L, gamma, rho_inf, p_inf must be positive (gamma > 1)");
  if (c->nvort < 0 || c->nvort > 16 || (c->nvort > 0 && !c->vort))
    return set_error(err, FR_EINVAL, "nvort must be in 0..16 with a vortex array");
  if (c->indicator < 0 || c->indicator > 3) return set_error(err, FR_EINVAL, "bad indicator");
  if (c->precision < 0 || c->precision > 4) return set_error(err, FR_EINVAL, "precision must be 0..4");
  if ((c->precision == 2 || c->precision == 3) && !(c->dim == 3 && c->p == 3))
    return set_error(err, FR_EINVAL, "the tensor-core operator forms (precision 2, 3) are built for 3D p = 3");
  if (!(c->dt > 0) && !(c->cfl > 0)) return set_error(err, FR_EINVAL, "need dt > 0 or cfl > 0");
  return 0;
}

// Issues the connectivity and face lists of `keys` into the mesh's tables: the leaf count is
// *d_n on the device (at most n_ub) or exactly n_ub (d_n null).  The packed face-list counts go
// to *d_faces and a 2:1 violation to bad[0]; `hcon` receives the per-hanging-face contributors.
// append: *d_faces holds zero and the connectivity kernel appends the faces to the lists itself
// (one launch; the lists' order then varies from run to run, the fluxes do not); otherwise the
// lists are written in leaf order after a scan of the per-leaf counts.
// seq > 0 (append only): the kernel also publishes the mesh's ctlblk words to its mapped host words
// with this sequence number.
// X (append only): a sampled index of keys for the searches (tab null: none).
static int conn_issue(fr_mesh* m, const uint64_t* keys, int64_t n_ub, const int64_t* d_n, int64_t* d_faces,
                      int32_t* bad, Buf<int32_t>& hcon, bool append = false, int64_t seq = 0,
                      const KeyIndex& X = KeyIndex{}) {
  Err* err = &m->err;
  cudaStream_t s = m->stream;
  const int64_t S = n_ub * m->nfc;
  FR_TRY(m->nbr.ensure(m->A, S));
  FR_TRY(m->ftype.ensure(m->A, S));
  FR_TRY(m->slot.ensure(m->A, S));
  // the lists hold at most dim conforming and 2*dim hanging entries per element: allocate that
  // bound so the writes need no synchronisation
  if (append) {
    FR_TRY(m->conf.ensure(m->A, size_t(n_ub) * m->dim));
    FR_TRY(m->hang.ensure(m->A, size_t(n_ub) * m->nfc));
    FR_TRY(hcon.ensure(m->A, size_t(n_ub) * m->nfc * 4));
    FaceLists L;
    L.conf = m->conf.p;
    L.hang = m->hang.p;
    L.hcon = hcon.p;
    L.count = reinterpret_cast<unsigned long long*>(d_faces);
    L.index = X;
    if (seq > 0 && m->pub_d) {
      L.pub = m->pub_d;
      L.words = m->ctlblk.p;
      L.nwords = CTLBLK_WORDS;
      L.seq = seq;
      L.done = reinterpret_cast<unsigned long long*>(m->ctlblk.p + CTL_DONE);
    }
    return tree_conn(m->dim, m->g, keys, n_ub, d_n, m->nbr.p, m->ftype.p, m->slot.p, nullptr, bad, s, err,
                     nullptr, L);
  }
  FR_TRY(m->contrib.ensure(m->A, S * 4));
  Scratch Sc(&m->A);
  int64_t* cnt = Sc.get<int64_t>(n_ub);
  int64_t* off = Sc.get<int64_t>(n_ub);
  if (!cnt || !off) return set_error(err, FR_ENOMEM, "conn scratch");
  // connectivity and the per-leaf face-list counts in one kernel
  FR_TRY(tree_conn(m->dim, m->g, keys, n_ub, d_n, m->nbr.p, m->ftype.p, m->slot.p, m->contrib.p, bad, s, err, cnt));
  Offs O;
  FR_TRY(scan_counts64_local(cnt, off, n_ub, d_faces, Sc, s, err, &O));
  FR_TRY(m->conf.ensure(m->A, size_t(n_ub) * m->dim));
  FR_TRY(m->hang.ensure(m->A, size_t(n_ub) * m->nfc));
  FR_TRY(hcon.ensure(m->A, size_t(n_ub) * m->nfc * 4));
  if (m->dim == 2)
    launch_dependent(k_face_write<2>, nblk(n_ub), TB, s, static_cast<const int8_t*>(m->ftype.p),
                     static_cast<const int32_t*>(m->contrib.p), n_ub, d_n, O, m->conf.p, m->hang.p, hcon.p);
  else
    launch_dependent(k_face_write<3>, nblk(n_ub), TB, s, static_cast<const int8_t*>(m->ftype.p),
                     static_cast<const int32_t*>(m->contrib.p), n_ub, d_n, O, m->conf.p, m->hang.p, hcon.p);
  FR_LAUNCH_CHECK(err);
  return 0;
}

// Waits for the publication `seq` of the connectivity kernel (conn_issue) and copies the ctlblk
// words into h: a host spin on the mapped sequence word, with a stream query every 1024 reads
// (an error, or a finished stream without the publication, ends it) and a 60 s bound.
static int wait_published(fr_mesh* m, int64_t seq, int64_t* h) {
  const volatile int64_t* p = m->pub_h;
  const auto t0 = std::chrono::steady_clock::now();
  for (uint64_t it = 1;; ++it) {
    if (p[CTLBLK_WORDS] == seq) break;
    if ((it & 1023) == 0) {
      const cudaError_t q = cudaStreamQuery(m->stream);
      if (q == cudaSuccess) {
        if (p[CTLBLK_WORDS] == seq) break;
        return set_error(&m->err, FR_ECUDA, "adapt: the counts were not published");
      }
      if (q != cudaErrorNotReady) {
        cudaGetLastError();
        return set_error(&m->err, FR_ECUDA, "adapt read");
      }
      if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(60))
        return set_error(&m->err, FR_ECUDA, "adapt: no publication of the counts within 60 s");
    }
  }
  std::atomic_thread_fence(std::memory_order_acquire);
  for (int w = 0; w < CTLBLK_WORDS; ++w) h[w] = p[w];
  return 0;
}

// after the synchronisation: the flags of conn_issue and the mapping (bad[0] 2:1 violation,
// bad[1] a new leaf the mapping could not place)
static int conn_check(fr_mesh* m, const int32_t* hb) {
  if (hb[0]) return set_error(&m->err, FR_EINVAL, "tree is not 2:1 balanced (connectivity)");
  if (hb[1])
    return set_error(&m->err, FR_EINVAL, "mapping found a new leaf that is neither kept, refined nor fused");
  return 0;
}

// after conn_check: keeps the face-list counts and the per-hanging-face contributor table
static int conn_finish(fr_mesh* m, int64_t faces, const int32_t* hb, Buf<int32_t>& hcon) {
  FR_TRY(conn_check(m, hb));
  m->n_conf = faces & 0xFFFFFFFFll;
  m->n_hang = faces >> 32;
  Buf<int32_t> old = m->contrib;  // the per element-face table is not needed after the lists
  m->contrib = hcon;
  hcon = Buf<int32_t>{};
  old.release(m->A);
  return 0;
}

// connectivity and face lists of the current tree (one host synchronisation)
int rebuild_conn(fr_mesh* m) {
  Err* err = &m->err;
  cudaStream_t s = m->stream;
  Scratch Sc(&m->A);
  int32_t* bad = Sc.get<int32_t>(2);
  int64_t* tot = Sc.get<int64_t>(1);
  if (!bad || !tot) return set_error(err, FR_ENOMEM, "conn scratch");
  FR_CUDA(err, cudaMemsetAsync(bad, 0, 8, s));
  Buf<int32_t> hcon;
  int rc = conn_issue(m, m->keys.p, m->M, nullptr, tot, bad, hcon);
  int64_t h = 0;
  int32_t hb[2] = {0, 0};
  if (!rc && (cudaMemcpyAsync(&h, tot, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
              cudaMemcpyAsync(hb, bad, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
              cudaStreamSynchronize(s) != cudaSuccess))
    rc = set_error(err, FR_ECUDA, "conn read");
  if (!rc) rc = conn_finish(m, h, hb, hcon);
  hcon.release(m->A);
  return rc;
}

int ensure_state(fr_mesh* m, int64_t M) {
  FR_TRY(m->u.ensure(m->A, size_t(M) * m->EU));
  FR_TRY(m->w.ensure(m->A, size_t(M) * m->EU));
  FR_TRY(m->trace.ensure(m->A, size_t(M) * m->EF));
  FR_TRY(m->fcomm.ensure(m->A, size_t(M) * m->EF));
  FR_TRY(m->flags.ensure(m->A, size_t(M)));
  return 0;
}

// traces of the current state (mask: only of the elements with a non-zero entry, the others
// already hold theirs)
int refresh_traces(fr_mesh* m, const int8_t* mask = nullptr) {
  m->traces_ok = false;
  FR_TRY(launch_traces(m->cfg.precision, m->dim, m->p, m->u.p, m->M, m->ops, m->trace.p, m->stream, &m->err, mask));
  m->traces_ok = true;
  return 0;
}

// The time-step buffers of the current tree.  An allocation that fails late in an adaptation or a
// state upload can leave them missing or short (Buf::ensure releases a block before it allocates
// the larger one); they are grown again here, and the traces recomputed, before anything reads
// them, so a failed call leaves the mesh usable.
int ready_buffers(fr_mesh* m) {
  const size_t M = size_t(m->M);
  if (!m->u.p || m->u.cap < M * m->EU || !m->keys.p || m->keys.cap < M)
    return set_error(&m->err, FR_EINVAL, "the mesh lost its state in an earlier failed call");
  FR_TRY(m->w.ensure(m->A, M * m->EU));
  FR_TRY(m->fcomm.ensure(m->A, M * m->EF));
  FR_TRY(m->flags.ensure(m->A, M));
  if (!m->trace.p || m->trace.cap < M * m->EF) {
    m->traces_ok = false;
    FR_TRY(m->trace.ensure(m->A, M * m->EF));
  }
  if (!m->traces_ok) FR_TRY(refresh_traces(m));
  return 0;
}

FaceArgs face_args(fr_mesh* m) {
  FaceArgs A{};
  A.trace = m->trace.p;
  A.fcomm = m->fcomm.p;
  A.nbr = m->nbr.p;
  A.conf = m->conf.p;
  A.hang = m->hang.p;
  A.contrib = m->contrib.p;
  A.n_conf = m->n_conf;
  A.n_hang = m->n_hang;
  A.gamma = m->cfg.gamma;
  return A;
}

int stage(fr_mesh* m, const double* us, const double* un, double* out, double a, double b, double c,
          bool traces, int8_t* flags = nullptr) {
  cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
  const bool rec = m->prof && (m->prof_count++ % m->prof_stride) == 0;
  if (rec) {
    e0 = m->next_event();
    e1 = m->next_event();
    e2 = m->next_event();
    cudaEventRecord(e0, m->stream);
  }
  FR_TRY(launch_faces(m->cfg.precision, m->dim, m->p, face_args(m), m->ops, m->stream, &m->err));
  if (rec) {
    cudaEventRecord(e1, m->stream);
    int64_t nsub = int64_t(1) << (m->dim - 1);
    m->recs.push_back({0, e0, e1, (m->n_conf + m->n_hang * nsub) * m->Nf});
  }
  StageArgs S{};
  S.keys = m->keys.p;
  S.us = us;
  S.un = un;
  S.fcomm = m->fcomm.p;
  S.out = out;
  S.trace_out = traces ? m->trace.p : nullptr;
  S.M = m->M;
  S.g = m->g;
  S.twoL = 2.0 / m->cfg.L;
  S.gamma = m->cfg.gamma;
  S.a = a;
  S.b = b;
  S.c = c;
  S.rk = rk_mode(a, b);
  S.status = m->status;
  S.flags = flags;
  S.th_r = m->cfg.th_refine;
  S.th_c = m->cfg.th_coarsen;
  FR_TRY(launch_stage(m->cfg.precision, m->dim, m->p, S, m->ops, m->stream, &m->err));
  if (rec) {
    cudaEventRecord(e2, m->stream);
    m->recs.push_back({1, e1, e2, m->M * m->N});
  }
  return 0;
}

// one SSP-RK3 step (Eq. rk3): u1 = u + dt R(u); u2 = 3/4 u + 1/4 u1 + 1/4 dt R(u1);
// u^{n+1} = 1/3 u + 2/3 u2 + 2/3 dt R(u2).  Buffers: u holds u^n, w holds u1 then u2.
// In the FP64 form with the density-gradient indicator, a step that ends on a multiple of
// adapt_every also writes the flags of the new state from its last element kernel (the indicator
// kernel of the next adaptation is then skipped).
int rk3_step(fr_mesh* m) {
  double dt = m->dt;
  m->flags_fresh = false;
  const bool want = m->cfg.precision == 0 && m->cfg.indicator == 0 && m->cfg.adapt_every > 0 &&
                    (m->step + 1) % m->cfg.adapt_every == 0;
  FR_TRY(stage(m, m->u.p, nullptr, m->w.p, 0.0, 1.0, dt, true));
  FR_TRY(stage(m, m->w.p, m->u.p, m->w.p, 0.75, 0.25, 0.25 * dt, true));
  FR_TRY(stage(m, m->w.p, m->u.p, m->u.p, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0 * dt, true, want ? m->flags.p : nullptr));
  m->flags_fresh = want;
  m->t += dt;
  m->step += 1;
  return 0;
}

int compute_flags(fr_mesh* m, double* eta) {
  if (m->cfg.indicator == 2) {
    FR_CUDA(&m->err, cudaMemsetAsync(m->flags.p, 0, size_t(m->M), m->stream));
    return 0;
  }
  if (m->cfg.indicator == 3 && m->mlp_n > 0 && !eta) {
    // learned indicator: features of the current state, then the MLP's argmax
    int in = mlp_in_dim(m->dim);
    Scratch Sc(&m->A);
    void* X = Sc.get<uint16_t>(size_t(m->M) * in);
    if (!X) return set_error(&m->err, FR_ENOMEM, "feature scratch");
    FR_TRY(mlp_features(m->dim, m->p, m->u.p, m->keys.p, m->M, m->g, m->cfg.Dbase, m->cfg.gamma,
                        m->ops, X, m->stream, &m->err));
    return mlp_forward(m->mlp_params.p, in, X, m->M, nullptr, m->flags.p, m->status, m->stream, &m->err);
  }
  // flags the last time step already wrote for the current state
  if (m->cfg.indicator == 0 && !eta && m->flags_fresh) return 0;
  // density gradient (indicator 0, and the fallback of the learned indicator) or analytic centre
  return launch_indicator(m->dim, m->p, m->cfg.indicator == 1 ? 1 : 0, m->cfg.th_refine, m->cfg.th_coarsen,
                          m->t, m->keys.p, m->M, m->g, m->prob, m->ops, m->u.p, m->flags.p, eta,
                          m->stream, &m->err);
}

struct Timer {
  cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
  bool on;
  cudaStream_t s;
  Timer(bool enable, cudaStream_t st) : on(enable), s(st) {
    if (on)
      for (auto& x : e) cudaEventCreate(&x);
  }
  ~Timer() {
    if (on)
      for (auto& x : e) cudaEventDestroy(x);
  }
  void mark(int k) {
    if (on) cudaEventRecord(e[k], s);
  }
  double ms(int a, int b) {
    if (!on) return 0.0;
    float v = 0.f;
    cudaEventSynchronize(e[b]);
    cudaEventElapsedTime(&v, e[a], e[b]);
    return double(v);
  }
};

// Adaptation: edit the tree with the flags, balance, and (if `transfer`) carry the state over.
// Adaptations of meshes up to this many leaves (times 2^dim, plus the balance passes' octant
// capacity) are issued without host synchronisations until the connectivity counts are read:
// below it launch and synchronisation latency, not the kernels, set the cost of an adaptation.
constexpr int64_t FAST_ADAPT_MAX = int64_t(1) << 20;

int adapt_impl(fr_mesh* m, const int8_t* d_flags, fr_adapt_stats* st, bool transfer) {
  Err* err = &m->err;
  cudaStream_t s = m->stream;
  Timer T(st != nullptr, s);
  T.mark(0);
  const int8_t* fl = d_flags;
  if (!fl) {
    FR_TRY(compute_flags(m, nullptr));
    fl = m->flags.p;
  }
  const int Dlow = m->cfg.Dbase + 2;
  const int64_t M0 = m->M;
  int64_t n_ub = M0 << m->dim;
  bool fast = transfer && n_ub + int64_t(m->g.Dmax) * 4096 <= FAST_ADAPT_MAX;
  int64_t* ctl = m->ctlblk.p;
  int32_t* bad = reinterpret_cast<int32_t*>(ctl + CTLBLK_BAD);
  int64_t h_ctl[CTLBLK_WORDS] = {0};
  int32_t hb[2] = {0, 0}, hs = 0;
  Buf<uint64_t> nk;
  Buf<double> nu;
  Buf<int32_t> src, hcon;
  Buf<int8_t> tag;
  Buf<double> ntr;
  // sampled indexes of the edited and balanced trees (issued without synchronisation): the edit
  // writes the first, each balance pass the next, and the searches of the passes and of the
  // connectivity read them
  Buf<uint64_t> tabA, tabB;
  KeyIndex X;
  bool conn_dirty = false;  // the mesh's connectivity tables now describe the new tree
  // the traces of unchanged elements are carried over by the transfer (when the current ones are
  // valid), which also computes those of the refined and fused elements from their new state
  const bool carry = transfer && m->traces_ok;
  // issued without synchronisation, the edit and the balance passes carry each new leaf's origin
  // in the old tree (src) and its relation to it (tag): the old->new mapping of Sec. 4.2 without a
  // search
  if (fast) {
    int passes = 0;
    for (int D = m->g.Dmax; D >= Dlow && D >= 2; --D) ++passes;
    X.sh = key_index_shift(n_ub + int64_t(passes) * 4096);
    const size_t nt = size_t(((n_ub + int64_t(passes) * 4096) >> X.sh) + 1);
    int r0 = tabA.ensure(m->A, nt);
    if (!r0) r0 = tabB.ensure(m->A, nt);
    if (r0) {  // nothing of the mesh has changed yet
      tabA.release(m->A);
      tabB.release(m->A);
      return r0;
    }
    X.tab = tabA.p;
  }
  int rc = tree_edit(m->dim, m->g, m->cfg.Dbase, m->keys.p, fl, M0, nk, ctl, bad, m->A, s, err,
                     fast ? &src : nullptr, fast ? &tag : nullptr, X);
  // map, transfer and connectivity of the new tree nk (leaf count *d_n, at most nb)
  auto rest = [&](int64_t nb, const int64_t* d_n) -> int {
    int r = 0;
    if (transfer) {
      // large meshes (and a fast path that fell back to exact sizes) map the new leaves with one
      // search per leaf; otherwise src and tag came with the balanced tree
      if (!fast) {
        if (!r) r = src.ensure(m->A, nb);
        if (!r) r = tag.ensure(m->A, nb);
        if (!r) r = tree_map(m->dim, m->g, m->keys.p, M0, nk.p, nb, d_n, src.p, tag.p, bad + 1, s, err);
      }
      T.mark(1);
      if (!r) r = nu.ensure(m->A, size_t(nb) * m->EU);
      TraceCopy tc{};
      if (!r && carry) {
        r = ntr.ensure(m->A, size_t(nb) * m->EF);
        tc = TraceCopy{m->trace.p, ntr.p, trace_kind(m->cfg.precision), m->EF * trace_elem_bytes(m->cfg.precision)};
      }
      if (!r)
        r = launch_transfer(m->dim, m->p, m->g, m->keys.p, M0, nk.p, src.p, tag.p, bad + 1, nb, d_n, m->ops, m->u.p,
                            nu.p, tc, s, err);
    } else {
      T.mark(1);
    }
    T.mark(2);
    int64_t seq = 0;
    if (!r) {
      conn_dirty = true;
      // issued without synchronisation: the edit's first kernel zeroed the face counter and the
      // finished-block counter; the last block publishes the counts to mapped host memory
      seq = (fast && m->pub_h) ? ++m->pub_seq : 0;
      r = conn_issue(m, nk.p, nb, d_n, ctl + CTL_FACES, bad, hcon, fast, seq, fast ? X : KeyIndex{});
    }
    // one read: the control block, the error flags and the status word are adjacent
    if (!r && seq > 0) {
      r = wait_published(m, seq, h_ctl);
    } else if (!r && (cudaMemcpyAsync(h_ctl, ctl, sizeof(h_ctl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                      cudaStreamSynchronize(s) != cudaSuccess)) {
      r = set_error(err, FR_ECUDA, "adapt read");
    }
    if (!r) {
      std::memcpy(hb, &h_ctl[CTLBLK_BAD], sizeof(hb));
      std::memcpy(&hs, &h_ctl[CTLBLK_STATUS], sizeof(hs));
    }
    if (!r && hs) {
      r = set_error(err, FR_ETIMEOUT, "a tensor-core completion wait gave up (indicator or element kernel)");
      // reported once: the status word starts clear for the next call
      if (cudaMemsetAsync(m->status, 0, 4, s) != cudaSuccess) cudaGetLastError();
    }
    return r;
  };
  int exact_depth = 0;  // the first balance pass run with exact sizes (0: none)
  if (!rc && fast) {
    int nslot = CTL_N;  // the slot that holds the balanced tree's leaf count
    rc = tree_balance_async(m->dim, m->g, Dlow, nk, ctl, &n_ub, m->A, s, err, &src, &tag, &nslot, &X,
                            X.tab ? tabB.p : nullptr);
    if (!rc) rc = rest(n_ub, ctl + nslot);
    if (!rc) h_ctl[CTL_N] = h_ctl[nslot];
    if (!rc && h_ctl[CTL_OVER] != 0) {
      // a balance pass generated more octants than the issued passes hold: finish the balance
      // from that depth with exact sizes (from the count in CTL_N) and redo the rest
      const int Dov = int(h_ctl[CTL_OVER]);
      if (cudaMemsetAsync(ctl + CTL_OVER, 0, 8, s) != cudaSuccess || cudaMemsetAsync(bad, 0, 8, s) != cudaSuccess ||
          (nslot != CTL_N &&
           cudaMemcpyAsync(ctl + CTL_N, ctl + nslot, 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess))
        rc = set_error(err, FR_ECUDA, "memset");
      if (!rc) rc = tree_balance(m->dim, m->g, Dov, Dlow, nk, ctl, n_ub, h_ctl, m->A, s, err);
      exact_depth = Dov;
      hcon.release(m->A);
      fast = false;
    }
  } else if (!rc) {
    rc = tree_balance(m->dim, m->g, m->g.Dmax, Dlow, nk, ctl, n_ub, h_ctl, m->A, s, err);
    if (m->g.Dmax >= Dlow && m->g.Dmax >= 2) exact_depth = m->g.Dmax;
  }
  if (!rc && !fast) rc = rest(h_ctl[CTL_N], nullptr);
  if (!rc) rc = conn_check(m, hb);
  const int64_t M1 = h_ctl[CTL_N];
  src.release(m->A);
  tag.release(m->A);
  tabA.release(m->A);
  tabB.release(m->A);
  if (!rc) {
    // the time-step buffers for the new size, while the mesh still holds the old tree (a block
    // that is released and not replaced here is grown again by ready_buffers)
    m->traces_ok = false;
    rc = m->w.ensure(m->A, size_t(M1) * m->EU);
    if (!rc && !carry) rc = m->trace.ensure(m->A, size_t(M1) * m->EF);
    if (!rc) rc = m->fcomm.ensure(m->A, size_t(M1) * m->EF);
    if (!rc) rc = m->flags.ensure(m->A, size_t(M1));
    if (!rc && !transfer) rc = m->u.ensure(m->A, size_t(M1) * m->EU);
  }
  if (rc) {
    // nothing of the mesh changed but the connectivity tables: rebuild them for the current tree
    // (keeping this call's error), so the mesh stays usable
    nk.release(m->A);
    nu.release(m->A);
    hcon.release(m->A);
    ntr.release(m->A);
    if (conn_dirty) {
      Err keep = *err;
      rebuild_conn(m);
      *err = keep;
    }
    return rc;
  }
  Buf<uint64_t> ok = m->keys;
  m->keys = nk;
  ok.release(m->A);
  m->M = M1;
  if (transfer) {
    Buf<double> ou = m->u;
    m->u = nu;
    ou.release(m->A);
  }
  if (carry) {
    Buf<double> ot = m->trace;  // the carried traces become the mesh's
    m->trace = ntr;
    ntr = Buf<double>{};
    ot.release(m->A);
  }
  m->traces_ok = false;
  m->flags_fresh = false;
  rc = conn_finish(m, h_ctl[CTL_FACES], hb, hcon);
  hcon.release(m->A);
  if (!rc && carry) m->traces_ok = true;  // carried or computed by the transfer
  if (!rc && transfer && !carry) rc = refresh_traces(m);
  FR_TRY(rc);
  T.mark(3);
  if (st) {
    st->M_old = M0;
    st->M_new = M1;
    st->n_refined = h_ctl[CTL_REF];
    st->n_coarsened = h_ctl[CTL_COARSE];
    st->balance_passes = int(h_ctl[CTL_PASSES]);
    st->balance_exact_depth = exact_depth;
    st->ms_tree = T.ms(0, 1);
    st->ms_transfer = T.ms(1, 2);
    st->ms_conn = T.ms(2, 3);
  }
  return 0;
}

int set_exact(fr_mesh* m, double t) {
  m->flags_fresh = false;
  FR_TRY(launch_exact(m->dim, m->p, m->keys.p, m->M, m->g, t, m->prob, m->ops, m->u.p, m->stream, &m->err));
  m->t = t;
  return 0;
}

int init_impl(fr_mesh* m, const fr_config* cfg, const fr_allocator* alloc, void* stream) {
  Err* err = &m->err;
  FR_TRY(check_cfg(cfg, err));
  m->cfg = *cfg;
  m->vort.assign(cfg->vort, cfg->vort + 4 * cfg->nvort);
  m->cfg.vort = m->vort.data();
  m->dim = cfg->dim;
  m->p = cfg->p;
  m->n = cfg->p + 1;
  m->N = m->dim == 2 ? m->n * m->n : m->n * m->n * m->n;
  m->Nf = m->dim == 2 ? m->n : m->n * m->n;
  m->nv = m->dim + 2;
  m->nfc = 2 * m->dim;
  m->EU = m->nv * m->N;
  m->EF = m->nfc * m->nv * m->Nf;
  m->g = KG{cfg->Dmax, depth_bits(cfg->Dmax)};
  if (build_ops(m->p, &m->ops)) return set_error(err, FR_EINVAL, "operators");
  m->prob = DevProblem{};
  m->prob.L = cfg->L;
  m->prob.gamma = cfg->gamma;
  m->prob.rho_inf = cfg->rho_inf;
  m->prob.p_inf = cfg->p_inf;
  for (int a = 0; a < 3; ++a) m->prob.uinf[a] = cfg->uinf[a];
  m->prob.nvort = cfg->nvort;
  for (int k = 0; k < cfg->nvort; ++k)
    for (int j = 0; j < 4; ++j) m->prob.vort[k][j] = cfg->vort[4 * k + j];
  m->stream = static_cast<cudaStream_t>(stream);
  if (alloc) {
    m->user = *alloc;
    m->has_user = true;
  }
  m->A = Alloc{m->has_user ? &m->user : nullptr, m->stream, err, &m->cache};
  int devcount = 0;
  if (cudaGetDeviceCount(&devcount) != cudaSuccess || devcount == 0) {
    cudaGetLastError();
    return set_error(err, FR_ECUDA, "no CUDA device");
  }
  // uniform tree at Dbase, then passes of {closed form, flags, adapt}
  m->M = int64_t(1) << (m->dim * cfg->Dbase);
  FR_TRY(m->ctlblk.ensure(m->A, CTLBLK_WORDS));
  FR_CUDA(err, cudaMemsetAsync(m->ctlblk.p, 0, CTLBLK_WORDS * sizeof(int64_t), m->stream));
  m->status = reinterpret_cast<int32_t*>(m->ctlblk.p + CTLBLK_STATUS);
  {
    // without mapped host memory the adaptation reads its counts back by a copy instead
    void* hp = nullptr;
    void* dp = nullptr;
    if (cudaHostAlloc(&hp, (CTLBLK_WORDS + 1) * sizeof(int64_t), cudaHostAllocMapped) == cudaSuccess &&
        cudaHostGetDevicePointer(&dp, hp, 0) == cudaSuccess) {
      std::memset(hp, 0, (CTLBLK_WORDS + 1) * sizeof(int64_t));
      m->pub_h = static_cast<int64_t*>(hp);
      m->pub_d = static_cast<int64_t*>(dp);
    } else {
      if (hp) cudaFreeHost(hp);
      cudaGetLastError();
    }
  }
  FR_TRY(m->keys.ensure(m->A, m->M));
  FR_TRY(tree_uniform(m->dim, m->g, cfg->Dbase, m->keys.p, m->stream, err));
  FR_TRY(ensure_state(m, m->M));
  int passes = cfg->init_passes < 0 ? cfg->Dmax - cfg->Dbase : cfg->init_passes;
  for (int ps = 0; ps < passes; ++ps) {
    FR_TRY(set_exact(m, 0.0));
    if (cfg->indicator == 2) break;
    FR_TRY(compute_flags(m, nullptr));
    FR_TRY(adapt_impl(m, m->flags.p, nullptr, false));
  }
  FR_TRY(set_exact(m, 0.0));
  if (passes == 0 || cfg->indicator == 2) FR_TRY(rebuild_conn(m));
  FR_TRY(refresh_traces(m));
  if (cfg->dt > 0) {
    m->dt = cfg->dt;
  } else {
    FR_TRY(m->dmax.ensure(m->A, 1));
    FR_TRY(launch_maxspeed(m->dim, m->p, m->u.p, m->M, cfg->gamma, m->dmax.p, m->stream, err));
    unsigned long long bits = 0;
    FR_CUDA(err, cudaMemcpyAsync(&bits, m->dmax.p, 8, cudaMemcpyDeviceToHost, m->stream));
    FR_CUDA(err, cudaStreamSynchronize(m->stream));
    double smax;
    std::memcpy(&smax, &bits, 8);
    double hmin = cfg->L / double(int64_t(1) << cfg->Dmax);
    m->dt = cfg->cfl * hmin / ((2.0 * cfg->p + 1.0) * smax);
  }
  m->t = 0.0;
  m->step = 0;
  FR_CUDA(err, cudaStreamSynchronize(m->stream));
  return 0;
}

// the mapped host words, once the stream has finished (a kernel may still publish to them)
void free_pub(fr_mesh* m) {
  cudaStreamSynchronize(m->stream);
  if (m->pub_h) cudaFreeHost(m->pub_h);
  m->pub_h = m->pub_d = nullptr;
}

void free_all(fr_mesh* m) {
  m->keys.release(m->A);
  m->u.release(m->A);
  m->w.release(m->A);
  m->trace.release(m->A);
  m->fcomm.release(m->A);
  m->nbr.release(m->A);
  m->conf.release(m->A);
  m->hang.release(m->A);
  m->contrib.release(m->A);
  m->ftype.release(m->A);
  m->slot.release(m->A);
  m->flags.release(m->A);
  m->norm_part.release(m->A);
  m->norm_out.release(m->A);
  m->dmax.release(m->A);
  m->mlp_params.release(m->A);
  m->ctlblk.release(m->A);
  m->status = nullptr;
  m->A.release_cache();
  // blocks still handed out (none after a clean release) go back to the allocator as well
  auto live = m->cache.live;
  for (auto& b : live) m->A.put(b.first);
  m->A.release_cache();
}

int host_copy(Err* err, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind, cudaStream_t s) {
  if (bytes == 0) return 0;
  FR_CUDA(err, cudaMemcpyAsync(dst, src, bytes, kind, s));
  FR_CUDA(err, cudaStreamSynchronize(s));
  return 0;
}

KG geo_or_err(int dim, int Dmax, int* rc) {
  *rc = 0;
  if ((dim != 2 && dim != 3) || Dmax < 1 || Dmax > 30 || dim * Dmax + depth_bits(Dmax) > 63 ||
      (dim == 3 && Dmax > 19))
    *rc = set_error(global_err(), FR_EINVAL, "dim/Dmax out of range");
  return KG{Dmax, depth_bits(Dmax)};
}

}  // namespace

// =============================================================================================
extern "C" {

const char* fr_last_error(const fr_mesh* m) {
  return m ? m->err.msg.c_str() : global_err()->msg.c_str();
}

int fr_mesh_init(const fr_config* cfg, const fr_allocator* alloc, void* stream, fr_mesh** out) {
  if (!out) return set_error(global_err(), FR_EINVAL, "null output handle");
  *out = nullptr;
  fr_mesh* m = new fr_mesh();
  int rc = init_impl(m, cfg, alloc, stream);
  if (rc) {
    *global_err() = m->err;
    free_all(m);
    free_pub(m);
    delete m;
    return rc;
  }
  *out = m;
  return 0;
}

void fr_mesh_free(fr_mesh* m) {
  if (!m) return;
  free_all(m);
  free_pub(m);
  for (cudaEvent_t e : m->ev_pool) cudaEventDestroy(e);
  delete m;
}

int fr_step(fr_mesh* m, int nsteps, fr_step_stats* st) {
  if (!m || nsteps < 0) return set_error(m ? &m->err : global_err(), FR_EINVAL, "bad arguments");
  FR_TRY(ready_buffers(m));
  Timer T(st != nullptr, m->stream);
  T.mark(0);
  for (int k = 0; k < nsteps; ++k) FR_TRY(rk3_step(m));
  T.mark(1);
  if (st) {
    st->steps = nsteps;
    st->dof_updates = int64_t(nsteps) * m->M * m->N * m->nv;
    st->ms = T.ms(0, 1);
  }
  return 0;
}

int fr_run(fr_mesh* m, int nsteps, fr_step_stats* sst, fr_adapt_stats* ast) {
  if (!m || nsteps < 0) return set_error(m ? &m->err : global_err(), FR_EINVAL, "bad arguments");
  fr_step_stats acc{};
  fr_adapt_stats aacc{};
  for (int k = 0; k < nsteps; ++k) {
    fr_step_stats one{};
    FR_TRY(fr_step(m, 1, sst ? &one : nullptr));
    acc.steps += one.steps;
    acc.dof_updates += one.dof_updates;
    acc.ms += one.ms;
    if (m->cfg.adapt_every > 0 && m->step % m->cfg.adapt_every == 0) {
      fr_adapt_stats a{};
      FR_TRY(adapt_impl(m, nullptr, ast ? &a : nullptr, true));
      aacc.M_old = a.M_old;
      aacc.M_new = a.M_new;
      aacc.n_refined += a.n_refined;
      aacc.n_coarsened += a.n_coarsened;
      aacc.balance_passes += a.balance_passes;
      if (a.balance_exact_depth > aacc.balance_exact_depth) aacc.balance_exact_depth = a.balance_exact_depth;
      aacc.ms_tree += a.ms_tree;
      aacc.ms_transfer += a.ms_transfer;
      aacc.ms_conn += a.ms_conn;
    }
  }
  if (sst) *sst = acc;
  if (ast) *ast = aacc;
  return 0;
}

int fr_adapt(fr_mesh* m, const int8_t* dev_flags, fr_adapt_stats* st) {
  if (!m) return set_error(global_err(), FR_EINVAL, "null mesh");
  FR_TRY(ready_buffers(m));
  return adapt_impl(m, dev_flags, st, true);
}

int fr_flags(fr_mesh* m, int8_t* host_flags, double* host_eta, int64_t cap) {
  if (!m) return set_error(global_err(), FR_EINVAL, "null mesh");
  if (cap < m->M) return set_error(&m->err, FR_EOVERFLOW, "capacity below M");
  FR_TRY(ready_buffers(m));
  Buf<double> eta;
  if (host_eta) FR_TRY(eta.ensure(m->A, m->M));
  if (m->cfg.indicator == 2) {
    FR_CUDA(&m->err, cudaMemsetAsync(m->flags.p, 0, size_t(m->M), m->stream));
    if (host_eta) FR_CUDA(&m->err, cudaMemsetAsync(eta.p, 0, size_t(m->M) * 8, m->stream));
  } else {
    FR_TRY(compute_flags(m, host_eta ? eta.p : nullptr));
  }
  int rc = host_copy(&m->err, host_flags, m->flags.p, size_t(m->M), cudaMemcpyDeviceToHost, m->stream);
  if (!rc && host_eta)
    rc = host_copy(&m->err, host_eta, eta.p, size_t(m->M) * 8, cudaMemcpyDeviceToHost, m->stream);
  eta.release(m->A);
  return rc;
}

int fr_rhs(fr_mesh* m, double* host_R, int64_t cap) {
  if (!m) return set_error(global_err(), FR_EINVAL, "null mesh");
  int64_t S = m->M * m->EU;
  if (cap < S) return set_error(&m->err, FR_EOVERFLOW, "capacity below M*nv*N");
  FR_TRY(ready_buffers(m));
  FR_TRY(stage(m, m->u.p, nullptr, m->w.p, 0.0, 0.0, 1.0, false));
  return host_copy(&m->err, host_R, m->w.p, size_t(S) * 8, cudaMemcpyDeviceToHost, m->stream);
}

int fr_norms(fr_mesh* m, fr_norms_out* out) {
  if (!m || !out) return set_error(m ? &m->err : global_err(), FR_EINVAL, "null argument");
  int64_t nb = norms_blocks(m->dim, m->p, m->M);
  FR_TRY(m->norm_part.ensure(m->A, size_t(nb + 1) * 8));
  FR_TRY(m->norm_out.ensure(m->A, 8));
  FR_TRY(launch_norms(m->dim, m->p, m->keys.p, m->M, m->g, m->t, m->prob, m->ops, m->u.p,
                      m->norm_part.p, nb + 1, m->norm_out.p, m->stream, &m->err));
  double h[8];
  FR_TRY(host_copy(&m->err, h, m->norm_out.p, 64, cudaMemcpyDeviceToHost, m->stream));
  out->t = m->t;
  out->l2_rho = std::sqrt(h[0]);
  for (int v = 0; v < 5; ++v) out->integral[v] = v < m->nv ? h[1 + v] : 0.0;
  out->min_rho = h[m->nv + 1];
  out->min_p = h[m->nv + 2];
  out->M = m->M;
  return 0;
}

int fr_get_leaves(fr_mesh* m, uint64_t* host_keys, int64_t cap, int64_t* M) {
  if (!m) return set_error(global_err(), FR_EINVAL, "null mesh");
  if (M) *M = m->M;
  if (!host_keys) return 0;
  if (cap < m->M) return set_error(&m->err, FR_EOVERFLOW, "capacity below M");
  return host_copy(&m->err, host_keys, m->keys.p, size_t(m->M) * 8, cudaMemcpyDeviceToHost, m->stream);
}

int fr_get_state(fr_mesh* m, double* host_u, int64_t cap) {
  if (!m) return set_error(global_err(), FR_EINVAL, "null mesh");
  int64_t S = m->M * m->EU;
  if (cap < S) return set_error(&m->err, FR_EOVERFLOW, "capacity below M*nv*N");
  return host_copy(&m->err, host_u, m->u.p, size_t(S) * 8, cudaMemcpyDeviceToHost, m->stream);
}

int fr_set_state(fr_mesh* m, const uint64_t* host_keys, int64_t M, const double* host_u) {
  if (!m) return set_error(global_err(), FR_EINVAL, "null mesh");
  if (M <= 0 || !host_keys || !host_u) return set_error(&m->err, FR_EINVAL, "bad arguments");
  Err* err = &m->err;
  cudaStream_t s = m->stream;
  // keys and state are copied in, the keys validated and the connectivity built, with one
  // synchronisation; the state lands in the stage buffer, so the current one survives a rejection
  Buf<uint64_t> nk;
  Buf<int32_t> hcon;
  Scratch Sc(&m->A);
  int32_t* bad = Sc.get<int32_t>(3);  // [0] 2:1 violation, [1] (mapping, unused here), [2] invalid tree
  int64_t* tot = Sc.get<int64_t>(1);
  if (!bad || !tot) return set_error(err, FR_ENOMEM, "set_state scratch");
  FR_TRY(nk.ensure(m->A, M));
  FR_TRY(m->w.ensure(m->A, size_t(M) * m->EU));
  int rc = 0;
  if (cudaMemcpyAsync(nk.p, host_keys, size_t(M) * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(m->w.p, host_u, size_t(M) * m->EU * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(bad, 0, 12, s) != cudaSuccess)
    rc = set_error(err, FR_ECUDA, "set_state copies");
  if (!rc) rc = tree_validate_async(m->dim, m->g, nk.p, M, m->cfg.Dbase, m->cfg.Dmax, bad + 2, s, err);
  if (!rc) rc = conn_issue(m, nk.p, M, nullptr, tot, bad, hcon);
  int64_t h = 0;
  int32_t hb[3] = {0, 0, 0};
  if (!rc && (cudaMemcpyAsync(&h, tot, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
              cudaMemcpyAsync(hb, bad, 12, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
              cudaStreamSynchronize(s) != cudaSuccess))
    rc = set_error(err, FR_ECUDA, "set_state read");
  if (!rc && hb[2]) rc = set_error(err, FR_EINVAL, "keys are not a complete sorted linear tree in [Dbase, Dmax]");
  if (!rc && hb[0]) rc = set_error(err, FR_EINVAL, "tree is not 2:1 balanced (connectivity)");
  if (rc) {
    // the tables were overwritten for the rejected keys: rebuild them for the current tree
    nk.release(m->A);
    hcon.release(m->A);
    Err keep = *err;
    rebuild_conn(m);
    *err = keep;
    return rc;
  }
  Buf<uint64_t> old = m->keys;
  m->keys = nk;
  old.release(m->A);
  m->M = M;
  Buf<double> ou = m->u;  // the stage buffer holding the new state becomes the state
  m->u = m->w;
  m->w = ou;
  m->traces_ok = false;
  m->flags_fresh = false;
  rc = conn_finish(m, h, hb, hcon);
  hcon.release(m->A);
  FR_TRY(rc);
  FR_TRY(ensure_state(m, M));
  return refresh_traces(m);
}

int fr_get_conn(fr_mesh* m, int32_t* nbr, int8_t* ftype, int8_t* slot, int64_t cap) {
  if (!m) return set_error(global_err(), FR_EINVAL, "null mesh");
  int64_t S = m->M * m->nfc;
  if (cap < S) return set_error(&m->err, FR_EOVERFLOW, "capacity below M*2*dim");
  FR_TRY(host_copy(&m->err, nbr, m->nbr.p, size_t(S) * 4, cudaMemcpyDeviceToHost, m->stream));
  FR_TRY(host_copy(&m->err, ftype, m->ftype.p, size_t(S), cudaMemcpyDeviceToHost, m->stream));
  return host_copy(&m->err, slot, m->slot.p, size_t(S), cudaMemcpyDeviceToHost, m->stream);
}

int fr_set_exact(fr_mesh* m, double t) {
  if (!m) return set_error(global_err(), FR_EINVAL, "null mesh");
  FR_TRY(set_exact(m, t));
  return refresh_traces(m);
}

int fr_set_time(fr_mesh* m, double t) {
  if (!m) return set_error(global_err(), FR_EINVAL, "null mesh");
  m->t = t;
  return 0;
}

int fr_get_info(fr_mesh* m, fr_info* out) {
  if (!m || !out) return set_error(m ? &m->err : global_err(), FR_EINVAL, "null argument");
  out->t = m->t;
  out->dt = m->dt;
  out->M = m->M;
  out->step = m->step;
  out->dim = m->dim;
  out->p = m->p;
  out->nv = m->nv;
  out->N = m->N;
  out->n_conforming = m->n_conf;
  out->n_hanging = m->n_hang;
  return 0;
}

int fr_profile_enable(fr_mesh* m, int on) {
  if (!m) return set_error(global_err(), FR_EINVAL, "null mesh");
  FR_CUDA(&m->err, cudaStreamSynchronize(m->stream));
  m->prof = on != 0;
  m->prof_stride = on > 1 ? on : 1;
  m->prof_count = 0;
  m->recs.clear();
  m->ev_used = 0;
  m->launches0 = launch_counter();
  return 0;
}

int fr_profile_read(fr_mesh* m, fr_profile* out) {
  if (!m || !out) return set_error(m ? &m->err : global_err(), FR_EINVAL, "null argument");
  FR_CUDA(&m->err, cudaStreamSynchronize(m->stream));
  *out = fr_profile{};
  for (const auto& r : m->recs) {
    float ms = 0.f;
    FR_CUDA(&m->err, cudaEventElapsedTime(&ms, r.a, r.b));
    if (r.kind == 0) {
      out->face_launches += 1;
      out->face_ms += ms;
      out->face_points += r.points;
    } else {
      out->stage_launches += 1;
      out->stage_ms += ms;
      out->stage_points += r.points;
    }
  }
  out->kernel_launches = launch_counter() - m->launches0;
  return 0;
}

int64_t fr_kernel_launches(void) { return launch_counter(); }

// ---- learned adaptation indicator ----

int fr_mlp_param_count(int in_dim) {
  if (in_dim < 1 || in_dim > 4096) return set_error(global_err(), FR_EINVAL, "bad input width");
  return mlp_param_count(in_dim);
}

int fr_features(fr_mesh* m, void* d_X, int64_t cap, int32_t* in_dim) {
  if (!m) return set_error(global_err(), FR_EINVAL, "null mesh");
  int in = mlp_in_dim(m->dim);
  if (in_dim) *in_dim = in;
  if (!d_X) return 0;
  if (cap < m->M * in) return set_error(&m->err, FR_EOVERFLOW, "capacity below M*in_dim");
  FR_TRY(mlp_features(m->dim, m->p, m->u.p, m->keys.p, m->M, m->g, m->cfg.Dbase, m->cfg.gamma,
                      m->ops, d_X, m->stream, &m->err));
  FR_CUDA(&m->err, cudaStreamSynchronize(m->stream));
  return 0;
}

int fr_set_learned_indicator(fr_mesh* m, const float* host_params, int64_t n) {
  if (!m) return set_error(global_err(), FR_EINVAL, "null mesh");
  if (!host_params || n == 0) {
    m->mlp_n = 0;  // back to the density-gradient indicator
    return 0;
  }
  if (n != mlp_param_count(mlp_in_dim(m->dim)))
    return set_error(&m->err, FR_EINVAL, "parameter count does not match the feature width");
  FR_TRY(m->mlp_params.ensure(m->A, size_t(n)));
  FR_TRY(host_copy(&m->err, m->mlp_params.p, host_params, size_t(n) * 4, cudaMemcpyHostToDevice, m->stream));
  m->mlp_n = n;
  return 0;
}

int fr_mlp_forward(int in_dim, const float* d_params, const void* d_X, int64_t n, float* d_logits,
                   int8_t* d_flags, void* stream) {
  if (in_dim < 1 || in_dim > 64 || n < 0) return set_error(global_err(), FR_EINVAL, "bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Alloc A{nullptr, s, global_err()};
  Scratch S(&A);
  int* st = S.get<int>(1);
  if (!st) return set_error(global_err(), FR_ENOMEM, "scratch");
  FR_CUDA(global_err(), cudaMemsetAsync(st, 0, 4, s));
  FR_TRY(mlp_forward(d_params, in_dim, d_X, n, d_logits, d_flags, st, s, global_err()));
  int hs = 0;
  FR_CUDA(global_err(), cudaMemcpyAsync(&hs, st, 4, cudaMemcpyDeviceToHost, s));
  FR_CUDA(global_err(), cudaStreamSynchronize(s));
  if (hs) return set_error(global_err(), FR_ETIMEOUT, "a tensor-core completion wait gave up");
  return 0;
}

void fr_tc_set_wait_limit(long long cycles) { mlp_set_wait_cycles(cycles); }

int fr_mlp_grad(int in_dim, const float* d_params, const void* d_X, const int8_t* d_y, int64_t B,
                const float* class_w, float* d_grad, float* d_loss, void* stream) {
  if (in_dim < 1 || in_dim > 64 || B <= 0 || !class_w)
    return set_error(global_err(), FR_EINVAL, "bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Alloc A{nullptr, s, global_err()};
  FR_TRY(mlp_grad(d_params, in_dim, d_X, d_y, B, class_w, d_grad, d_loss, A, s, global_err()));
  FR_CUDA(global_err(), cudaStreamSynchronize(s));
  return 0;
}

int fr_mlp_train_step(int in_dim, float* d_params, float* d_m, float* d_v, int64_t step,
                      const void* d_X, const int8_t* d_y, int64_t B, const float* class_w, float lr,
                      float* d_loss, void* stream) {
  if (in_dim < 1 || in_dim > 64 || B <= 0 || !class_w || step < 0)
    return set_error(global_err(), FR_EINVAL, "bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Alloc A{nullptr, s, global_err()};
  FR_TRY(mlp_train_step(d_params, d_m, d_v, step, in_dim, d_X, d_y, B, class_w, lr, d_loss, A, s,
                        global_err()));
  return 0;
}

// ---- tree primitives on caller-owned device arrays ----

int fr_morton_encode(int dim, int Dmax, int64_t n, const int32_t* d_boxes, uint64_t* d_keys,
                     void* stream) {
  int rc;
  KG g = geo_or_err(dim, Dmax, &rc);
  if (rc) return rc;
  if (n < 0) return set_error(global_err(), FR_EINVAL, "n < 0");
  return tree_encode(dim, g, d_boxes, n, d_keys, static_cast<cudaStream_t>(stream), global_err());
}

int fr_keys_sort(int dim, int Dmax, uint64_t* d_keys, int64_t n, void* stream) {
  int rc;
  KG g = geo_or_err(dim, Dmax, &rc);
  if (rc) return rc;
  if (n < 0) return set_error(global_err(), FR_EINVAL, "n < 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Alloc A{nullptr, s, global_err()};
  Scratch S(&A);
  uint64_t* tmp = S.get<uint64_t>(n);
  if (!tmp) return set_error(global_err(), FR_ENOMEM, "sort scratch");
  FR_TRY(radix_sort_keys(d_keys, tmp, n, dim * Dmax + g.mb, S, s, global_err()));
  FR_CUDA(global_err(), cudaStreamSynchronize(s));
  return 0;
}

int fr_keys_linearise(int dim, int Dmax, const uint64_t* d_keys, int64_t n, uint64_t* d_out,
                      int64_t cap, int64_t* n_out, void* stream) {
  int rc;
  KG g = geo_or_err(dim, Dmax, &rc);
  if (rc) return rc;
  if (n < 0 || !n_out) return set_error(global_err(), FR_EINVAL, "bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Err* err = global_err();
  Alloc A{nullptr, s, err};
  Scratch S(&A);
  uint64_t* a = S.get<uint64_t>(n);
  uint64_t* tmp = S.get<uint64_t>(n);
  if (!a || !tmp) return set_error(err, FR_ENOMEM, "linearise scratch");
  if (n) FR_CUDA(err, cudaMemcpyAsync(a, d_keys, size_t(n) * 8, cudaMemcpyDeviceToDevice, s));
  FR_TRY(radix_sort_keys(a, tmp, n, dim * Dmax + g.mb, S, s, err));
  Buf<uint64_t> out;
  int64_t m = 0;
  rc = tree_linearise(dim, g, a, n, out, &m, A, s, err);
  *n_out = m;
  if (!rc && m > cap) rc = set_error(err, FR_EOVERFLOW, "output capacity too small");
  if (!rc && m) rc = cudaMemcpyAsync(d_out, out.p, size_t(m) * 8, cudaMemcpyDeviceToDevice, s) == cudaSuccess ? 0 : set_error(err, FR_ECUDA, "copy");
  out.release(A);
  if (!rc) FR_CUDA(err, cudaStreamSynchronize(s));
  return rc;
}

static int balance_or_adapt(int dim, int Dbase, int Dmax, const uint64_t* d_keys, const int8_t* d_flags,
                            int64_t n, uint64_t* d_out, int64_t cap, int64_t* n_out, void* stream) {
  int rc;
  KG g = geo_or_err(dim, Dmax, &rc);
  if (rc) return rc;
  if (n <= 0 || !n_out) return set_error(global_err(), FR_EINVAL, "bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Err* err = global_err();
  Alloc A{nullptr, s, err};
  bool ok = false;
  FR_TRY(tree_validate(dim, g, d_keys, n, 0, Dmax, &ok, A, s, err));
  if (!ok) return set_error(err, FR_EINVAL, "input is not a complete sorted linear tree");
  Buf<uint64_t> k;
  Scratch S(&A);
  int64_t* ctl = S.get<int64_t>(CTL_SLOTS);
  if (!ctl) return set_error(err, FR_ENOMEM, "scratch");
  int64_t h_ctl[CTL_SLOTS] = {n};
  int64_t n_ub = n;
  if (d_flags) {
    rc = tree_edit(dim, g, Dbase, d_keys, d_flags, n, k, ctl, nullptr, A, s, err);
    n_ub = n << dim;
  } else {
    rc = k.ensure(A, n);
    if (!rc) rc = cudaMemcpyAsync(k.p, d_keys, size_t(n) * 8, cudaMemcpyDeviceToDevice, s) == cudaSuccess ? 0 : set_error(err, FR_ECUDA, "copy");
    if (!rc) rc = cudaMemcpyAsync(ctl, h_ctl, sizeof(h_ctl), cudaMemcpyHostToDevice, s) == cudaSuccess ? 0 : set_error(err, FR_ECUDA, "copy");
  }
  if (!rc) rc = tree_balance(dim, g, Dmax, d_flags ? Dbase + 2 : 2, k, ctl, n_ub, h_ctl, A, s, err);
  const int64_t m = h_ctl[CTL_N];
  *n_out = m;
  if (!rc && m > cap) rc = set_error(err, FR_EOVERFLOW, "output capacity too small");
  if (!rc) rc = cudaMemcpyAsync(d_out, k.p, size_t(m) * 8, cudaMemcpyDeviceToDevice, s) == cudaSuccess ? 0 : set_error(err, FR_ECUDA, "copy");
  k.release(A);
  if (!rc) FR_CUDA(err, cudaStreamSynchronize(s));
  return rc;
}

int fr_tree_balance(int dim, int Dmax, const uint64_t* d_keys, int64_t n, uint64_t* d_out,
                    int64_t cap, int64_t* n_out, void* stream) {
  return balance_or_adapt(dim, 0, Dmax, d_keys, nullptr, n, d_out, cap, n_out, stream);
}

int fr_tree_adapt(int dim, int Dbase, int Dmax, const uint64_t* d_keys, const int8_t* d_flags,
                  int64_t n, uint64_t* d_out, int64_t cap, int64_t* n_out, void* stream) {
  if (!d_flags) return set_error(global_err(), FR_EINVAL, "null flags");
  if (Dbase < 0 || Dbase > Dmax) return set_error(global_err(), FR_EINVAL, "Dbase out of range");
  return balance_or_adapt(dim, Dbase, Dmax, d_keys, d_flags, n, d_out, cap, n_out, stream);
}

int fr_tree_complete(int dim, int Dmin, int Dmax, double L, const double* d_pts, int64_t n,
                     uint64_t* d_out, int64_t cap, int64_t* n_out, void* stream) {
  int rc;
  KG g = geo_or_err(dim, Dmax, &rc);
  if (rc) return rc;
  if (n < 0 || !n_out || Dmin < 0 || Dmin > Dmax || !(L > 0))
    return set_error(global_err(), FR_EINVAL, "bad arguments");
  if (n > (int64_t(1) << 30)) return set_error(global_err(), FR_EINVAL, "too many points");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Err* err = global_err();
  Alloc A{nullptr, s, err};
  Buf<uint64_t> out;
  int64_t m = 0;
  rc = tree_complete(dim, g, Dmin, L, d_pts, n, out, &m, A, s, err);
  *n_out = m;
  if (!rc && m > cap) rc = set_error(err, FR_EOVERFLOW, "output capacity too small");
  if (!rc && m)
    rc = cudaMemcpyAsync(d_out, out.p, size_t(m) * 8, cudaMemcpyDeviceToDevice, s) == cudaSuccess
             ? 0 : set_error(err, FR_ECUDA, "copy");
  out.release(A);
  if (!rc) FR_CUDA(err, cudaStreamSynchronize(s));
  return rc;
}

int fr_tree_map(int dim, int Dmax, const uint64_t* d_old, int64_t n_old, const uint64_t* d_new,
                int64_t n_new, int32_t* d_src, int8_t* d_tag, void* stream) {
  int rc;
  KG g = geo_or_err(dim, Dmax, &rc);
  if (rc) return rc;
  if (n_old <= 0 || n_new < 0) return set_error(global_err(), FR_EINVAL, "bad sizes");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Err* err = global_err();
  Alloc A{nullptr, s, err};
  Scratch S(&A);
  int32_t* bad = S.get<int32_t>(1);
  if (!bad) return set_error(err, FR_ENOMEM, "map scratch");
  FR_CUDA(err, cudaMemsetAsync(bad, 0, 4, s));
  FR_TRY(tree_map(dim, g, d_old, n_old, d_new, n_new, nullptr, d_src, d_tag, bad, s, err));
  int32_t hb = 0;
  FR_CUDA(err, cudaMemcpyAsync(&hb, bad, 4, cudaMemcpyDeviceToHost, s));
  FR_CUDA(err, cudaStreamSynchronize(s));
  if (hb) return set_error(err, FR_EINVAL, "a new leaf is neither kept, refined nor fused");
  return 0;
}

int fr_tree_conn(int dim, int Dmax, const uint64_t* d_keys, int64_t n, int32_t* d_nbr,
                 int8_t* d_ftype, int8_t* d_slot, void* stream) {
  int rc;
  KG g = geo_or_err(dim, Dmax, &rc);
  if (rc) return rc;
  if (n <= 0) return set_error(global_err(), FR_EINVAL, "bad size");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Err* err = global_err();
  Alloc A{nullptr, s, err};
  bool ok = false;
  FR_TRY(tree_validate(dim, g, d_keys, n, 0, Dmax, &ok, A, s, err));
  if (!ok) return set_error(err, FR_EINVAL, "input is not a complete sorted linear tree");
  Scratch S(&A);
  int32_t* bad = S.get<int32_t>(1);
  if (!bad) return set_error(err, FR_ENOMEM, "conn scratch");
  FR_CUDA(err, cudaMemsetAsync(bad, 0, 4, s));
  FR_TRY(tree_conn(dim, g, d_keys, n, nullptr, d_nbr, d_ftype, d_slot, nullptr, bad, s, err));
  int32_t hb = 0;
  FR_CUDA(err, cudaMemcpyAsync(&hb, bad, 4, cudaMemcpyDeviceToHost, s));
  FR_CUDA(err, cudaStreamSynchronize(s));
  if (hb) return set_error(err, FR_EINVAL, "tree is not 2:1 balanced");
  return 0;
}

}  // extern "C"
