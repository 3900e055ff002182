// fr_oracle.cpp -- plain CPU oracle for h-adaptive FR on linear trees (arXiv 2306.06744).
//
// TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the benchmark's
// CPU-baseline leg, never by the GPU library or its Python binding.  It shares no code with the
// GPU library.  Each function names the passage of the paper it restates.  Where the paper is
// silent or garbled the reading taken is named in the comment ("reading: ...").
//
// Exact-result parts (keys, linearisation, balance, connectivity, mapping) are written as the
// plain definitions: set semantics, geometric containment and point location by predecessor
// search in the sorted key array.  Numerical parts (operators, FR residual, mortar, transfer,
// SSP-RK3, norms) are literal loops in FP64 with no sum factorisation or operator folding.
// Compiled with -ffp-contract=off so that results do not depend on the host's FMA use.

#include "fr_oracle.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <vector>

namespace {

thread_local std::string g_err;
int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

// ------------------------------------------------------------------------------------------
// Morton IDs (Sec. 2.2, Algorithm 1)
// ------------------------------------------------------------------------------------------

struct Geo {
  int dim, Dmax, mb;
};

// m_b = number of bits needed to write Dmax (Algorithm 1, step 1): ceil(log2(Dmax+1)).
int depth_bits(int Dmax) {
  int mb = 0;
  while ((1 << mb) < Dmax + 1) ++mb;
  return mb;
}

bool geo_ok(int dim, int Dmax) {
  if (dim != 2 && dim != 3) return false;
  if (Dmax < 1 || Dmax > 30) return false;
  return dim * Dmax + depth_bits(Dmax) <= 63;
}

struct Box {
  int depth;
  int64_t x[3];  // anchor (lowest corner, Sec. 2.2) in units of the finest cell, 0..2^Dmax-1
};

int64_t width(const Geo& g, int depth) { return int64_t(1) << (g.Dmax - depth); }

// Algorithm 1: interleave the depth-D coordinate bits, most significant level first, with the
// z bit above the y bit above the x bit inside one level (reading: x least significant, so the
// child index is x + 2y + 4z); pad dim*(Dmax-D) zeros; append D in m_b bits.
uint64_t encode(const Geo& g, const Box& b) {
  uint64_t raw = 0;
  for (int k = b.depth - 1; k >= 0; --k) {
    for (int a = g.dim - 1; a >= 0; --a) {
      uint64_t bit = (uint64_t(b.x[a]) >> (g.Dmax - b.depth + k)) & 1u;
      raw = (raw << 1) | bit;
    }
  }
  raw <<= g.dim * (g.Dmax - b.depth);
  return (raw << g.mb) | uint64_t(b.depth);
}

// Inverse of Algorithm 1 (Sec. 2.2: the anchor and width follow from the ID alone).
Box decode(const Geo& g, uint64_t key) {
  Box b{};
  b.depth = int(key & ((uint64_t(1) << g.mb) - 1));
  uint64_t raw = key >> g.mb;
  for (int a = 0; a < 3; ++a) b.x[a] = 0;
  for (int j = 0; j < g.Dmax; ++j)
    for (int a = 0; a < g.dim; ++a) b.x[a] |= int64_t((raw >> (j * g.dim + a)) & 1u) << j;
  return b;
}

bool key_valid(const Geo& g, uint64_t key) {
  int d = int(key & ((uint64_t(1) << g.mb) - 1));
  if (d > g.Dmax) return false;
  Box b = decode(g, key);
  for (int a = 0; a < g.dim; ++a)
    if (b.x[a] % width(g, d) != 0) return false;
  if ((key >> g.mb) >> (g.dim * g.Dmax)) return false;
  return encode(g, b) == key;
}

// Geometric containment: box A contains box B (A coarser or equal).
bool contains(const Geo& g, const Box& A, const Box& B) {
  if (A.depth > B.depth) return false;
  int64_t w = width(g, A.depth);
  for (int a = 0; a < g.dim; ++a)
    if (B.x[a] < A.x[a] || B.x[a] >= A.x[a] + w) return false;
  return true;
}

Box child_box(const Geo& g, const Box& A, int c) {
  Box C = A;
  C.depth = A.depth + 1;
  int64_t w = width(g, C.depth);
  for (int a = 0; a < g.dim; ++a) C.x[a] = A.x[a] + ((c >> a) & 1) * w;
  return C;
}

Box parent_box(const Geo& g, const Box& B) {
  Box P = B;
  P.depth = B.depth - 1;
  int64_t w = width(g, P.depth);
  for (int a = 0; a < g.dim; ++a) P.x[a] = (B.x[a] / w) * w;
  return P;
}

// Position of B inside its parent: bit a is set when B is the upper half along axis a.
int child_index(const Geo& g, const Box& B) {
  int c = 0;
  int64_t w = width(g, B.depth);
  for (int a = 0; a < g.dim; ++a) c |= int((B.x[a] / w) & 1) << a;
  return c;
}

int64_t wrap(const Geo& g, int64_t v) {
  int64_t n = int64_t(1) << g.Dmax;
  v %= n;
  return v < 0 ? v + n : v;
}

// Point location in a complete linear tree: the leaf that contains the finest cell at P is the
// largest key not above that cell's key (keys ascend in pre-order, Sec. 2.2).  Returns the index.
int64_t locate(const Geo& g, const std::vector<uint64_t>& keys, const int64_t P[3]) {
  Box cell{};
  cell.depth = g.Dmax;
  for (int a = 0; a < 3; ++a) cell.x[a] = a < g.dim ? P[a] : 0;
  uint64_t kc = encode(g, cell);
  auto it = std::upper_bound(keys.begin(), keys.end(), kc);
  if (it == keys.begin()) return -1;
  return int64_t(it - keys.begin()) - 1;
}

bool complete(const Geo& g, const std::vector<uint64_t>& keys) {
  // Complete and non-overlapping: sorted, every leaf begins where the previous one ended.
  int64_t next = 0;  // Morton index (in finest cells) of the next uncovered cell
  for (size_t i = 0; i < keys.size(); ++i) {
    if (!key_valid(g, keys[i])) return false;
    if (i && keys[i] <= keys[i - 1]) return false;
    Box b = decode(g, keys[i]);
    int64_t start = int64_t(keys[i] >> g.mb);
    if (start != next) return false;
    next = start + (int64_t(1) << (g.dim * (g.Dmax - b.depth)));
  }
  return next == (int64_t(1) << (g.dim * g.Dmax));
}

// ------------------------------------------------------------------------------------------
// Linearisation (Sec. 3.1): the leaves of a set of octants = drop duplicates and every octant
// that has a proper descendant in the set.
// ------------------------------------------------------------------------------------------
std::vector<uint64_t> linearise(const Geo& g, std::vector<uint64_t> v) {
  std::sort(v.begin(), v.end());
  v.erase(std::unique(v.begin(), v.end()), v.end());
  std::vector<uint64_t> out;
  for (size_t i = 0; i < v.size(); ++i) {
    Box A = decode(g, v[i]);
    // every octant whose anchor lies in A has a key in [lo, hi]
    uint64_t lo = (v[i] >> g.mb) << g.mb;
    uint64_t vol = uint64_t(1) << (g.dim * (g.Dmax - A.depth));
    uint64_t hi = ((((v[i] >> g.mb) + vol - 1)) << g.mb) | ((uint64_t(1) << g.mb) - 1);
    bool has_desc = false;
    for (auto it = std::lower_bound(v.begin(), v.end(), lo); it != v.end() && *it <= hi; ++it) {
      Box B = decode(g, *it);
      if (B.depth > A.depth && contains(g, A, B)) {
        has_desc = true;
        break;
      }
    }
    if (!has_desc) out.push_back(v[i]);
  }
  return out;
}

// ------------------------------------------------------------------------------------------
// Tree completion from scattered points (Sec. 3.1, construction algorithm; Sec. 5.1: a coarse
// background at Dmin, points encoded at Dmax).  Definition written out: starting from the root,
// an octant is split while its depth is below Dmin, or while it contains the finest cell of some
// point and is above Dmax; every other octant is a leaf.  Point cells: floor(x / L * 2^Dmax),
// clamped to the grid.
// ------------------------------------------------------------------------------------------
void complete_rec(const Geo& g, int Dmin, const std::set<uint64_t>& cells, const Box& o,
                  std::vector<uint64_t>& out) {
  bool split = o.depth < Dmin;
  if (!split && o.depth < g.Dmax) {
    // does o contain a point cell?  cells are depth-Dmax keys; those inside o lie in [lo, hi]
    uint64_t k = encode(g, o);
    uint64_t lo = (k >> g.mb) << g.mb;
    uint64_t vol = uint64_t(1) << (g.dim * (g.Dmax - o.depth));
    uint64_t hi = (((k >> g.mb) + vol - 1) << g.mb) | ((uint64_t(1) << g.mb) - 1);
    auto it = cells.lower_bound(lo);
    split = it != cells.end() && *it <= hi;
  }
  if (!split) {
    out.push_back(encode(g, o));
    return;
  }
  for (int c = 0; c < (1 << g.dim); ++c) complete_rec(g, Dmin, cells, child_box(g, o, c), out);
}

// ------------------------------------------------------------------------------------------
// 2:1 balance (Sec. 3.2).  Reading: strong (vertex) balance with periodic wrap; the result is the
// unique coarsest balanced refinement.  Definition written out: while some leaf A touches a leaf B
// more than one level finer, split A.  A coarser leaf A touches B iff A contains the anchor of one
// of B's 3^dim-1 same-size neighbour boxes.
// ------------------------------------------------------------------------------------------
std::vector<uint64_t> balance(const Geo& g, std::vector<uint64_t> keys) {
  std::sort(keys.begin(), keys.end());
  for (;;) {
    std::set<int64_t> split;
    for (size_t i = 0; i < keys.size(); ++i) {
      Box B = decode(g, keys[i]);
      int64_t w = width(g, B.depth);
      int nofs = g.dim == 2 ? 9 : 27;
      for (int o = 0; o < nofs; ++o) {
        int off[3] = {o % 3 - 1, (o / 3) % 3 - 1, g.dim == 3 ? o / 9 - 1 : 0};
        if (off[0] == 0 && off[1] == 0 && off[2] == 0) continue;
        int64_t P[3] = {0, 0, 0};
        for (int a = 0; a < g.dim; ++a) P[a] = wrap(g, B.x[a] + off[a] * w);
        int64_t j = locate(g, keys, P);
        if (decode(g, keys[j]).depth < B.depth - 1) split.insert(j);
      }
    }
    if (split.empty()) break;
    std::vector<uint64_t> next;
    for (size_t i = 0; i < keys.size(); ++i) {
      if (!split.count(int64_t(i))) {
        next.push_back(keys[i]);
        continue;
      }
      Box A = decode(g, keys[i]);
      for (int c = 0; c < (1 << g.dim); ++c) next.push_back(encode(g, child_box(g, A, c)));
    }
    std::sort(next.begin(), next.end());
    keys.swap(next);
  }
  return keys;
}

// ------------------------------------------------------------------------------------------
// Adaptation procedure (Sec. 4.1, adaptation algorithm), followed by 2:1 balance.
// Reading: refinement is ignored at Dmax and coarsening at or above Dbase; a leaf changes at most
// one level per adaptation.
// ------------------------------------------------------------------------------------------
std::vector<uint64_t> adapt_keys(const Geo& g, int Dbase, const std::vector<uint64_t>& keys,
                                 const int8_t* flags_in) {
  size_t M = keys.size();
  std::vector<int> flag(M);
  std::vector<Box> box(M);
  for (size_t i = 0; i < M; ++i) {
    box[i] = decode(g, keys[i]);
    flag[i] = flags_in[i];
    if (flag[i] > 0 && box[i].depth >= g.Dmax) flag[i] = 0;
    if (flag[i] < 0 && box[i].depth <= Dbase) flag[i] = 0;
  }
  std::set<uint64_t> leafset(keys.begin(), keys.end());
  std::map<uint64_t, int> flag_of;
  for (size_t i = 0; i < M; ++i) flag_of[keys[i]] = flag[i];
  // step 2: children of octants flagged for refinement are appended
  std::vector<uint64_t> T(keys.begin(), keys.end());
  for (size_t i = 0; i < M; ++i)
    if (flag[i] == 1)
      for (int c = 0; c < (1 << g.dim); ++c) T.push_back(encode(g, child_box(g, box[i], c)));
  // steps 3-4: a coarsening flag stands only if all 2^dim siblings are leaves flagged -1; their
  // parents are collected in P
  std::set<uint64_t> P;
  for (size_t i = 0; i < M; ++i) {
    if (flag[i] != -1) continue;
    Box par = parent_box(g, box[i]);
    bool all = true;
    for (int c = 0; c < (1 << g.dim) && all; ++c) {
      uint64_t s = encode(g, child_box(g, par, c));
      all = leafset.count(s) && flag_of[s] == -1;
    }
    if (all) P.insert(encode(g, par));
  }
  // step 5: remove the children of P, append P; step 6: sort and linearise
  std::vector<uint64_t> T2;
  for (uint64_t k : T) {
    Box b = decode(g, k);
    bool drop = false;
    if (b.depth > 0) drop = P.count(encode(g, parent_box(g, b))) > 0;
    if (!drop) T2.push_back(k);
  }
  for (uint64_t k : P) T2.push_back(k);
  T2 = linearise(g, T2);
  return balance(g, T2);
}

// ------------------------------------------------------------------------------------------
// Old -> new mapping (Sec. 4.2, mapping algorithm), by geometric containment.
// tag 0: same octant (copy); 1: the new leaf lies inside old leaf src (refined);
// 2: the new leaf contains old leaves, src is the first of them (fused).
// ------------------------------------------------------------------------------------------
void map_trees(const Geo& g, const std::vector<uint64_t>& old_keys,
               const std::vector<uint64_t>& new_keys, std::vector<int32_t>& src,
               std::vector<int8_t>& tag) {
  src.assign(new_keys.size(), -1);
  tag.assign(new_keys.size(), -1);
  for (size_t j = 0; j < new_keys.size(); ++j) {
    Box K = decode(g, new_keys[j]);
    int64_t i = locate(g, old_keys, K.x);
    Box A = decode(g, old_keys[i]);
    src[j] = int32_t(i);
    if (old_keys[i] == new_keys[j])
      tag[j] = 0;
    else if (contains(g, A, K))
      tag[j] = 1;
    else
      tag[j] = 2;
  }
}

// ------------------------------------------------------------------------------------------
// Face connectivity (Sec. 3.3, face connectivity algorithm), by point location.
// Reading of the missing figure: faces 0/1 = -x/+x, 2/3 = -y/+y, 4/5 = -z/+z; the matching face
// is f^1.  Contributor slot on a coarse face: the fine octant's child bits along the in-face
// axes, lower axis least significant (Sec. 3.3 worked example).
// ------------------------------------------------------------------------------------------
struct Conn {
  std::vector<int32_t> nbr;
  std::vector<int8_t> ftype, slot;
  std::vector<int32_t> contrib;  // [M][2dim][4]: coarse side contributors in slot order
};

int in_face_slot(const Geo& g, const Box& K, int axis) {
  int s = 0, sh = 0;
  int c = child_index(g, K);
  for (int b = 0; b < g.dim; ++b) {
    if (b == axis) continue;
    s |= ((c >> b) & 1) << sh;
    ++sh;
  }
  return s;
}

int build_conn(const Geo& g, const std::vector<uint64_t>& keys, Conn& cn) {
  size_t M = keys.size();
  int nf = 2 * g.dim, nsub = 1 << (g.dim - 1);
  cn.nbr.assign(M * nf, -1);
  cn.ftype.assign(M * nf, -1);
  cn.slot.assign(M * nf, -1);
  cn.contrib.assign(M * nf * 4, -1);
  for (size_t e = 0; e < M; ++e) {
    Box E = decode(g, keys[e]);
    int64_t w = width(g, E.depth);
    for (int f = 0; f < nf; ++f) {
      int axis = f / 2, side = f % 2;
      Box N = E;  // same-size box across the face (wrapped)
      N.x[axis] = wrap(g, E.x[axis] + (side ? w : -w));
      int64_t j = locate(g, keys, N.x);
      Box J = decode(g, keys[j]);
      size_t s = e * nf + f;
      if (J.depth == E.depth) {
        cn.nbr[s] = int32_t(j);
        cn.ftype[s] = 0;
      } else if (J.depth < E.depth) {
        if (J.depth != E.depth - 1) return fail(ORACLE_EINVAL, "tree is not 2:1 balanced");
        cn.nbr[s] = int32_t(j);
        cn.ftype[s] = 1;
        cn.slot[s] = int8_t(in_face_slot(g, E, axis));
      } else {
        // finer neighbours: the children of N that touch E's face
        cn.ftype[s] = 2;
        cn.slot[s] = 0;
        for (int c = 0; c < (1 << g.dim); ++c) {
          int bit_axis = (c >> axis) & 1;
          if (bit_axis != (side ? 0 : 1)) continue;
          Box C = child_box(g, N, c);
          int64_t k = locate(g, keys, C.x);
          if (keys[k] != encode(g, C)) return fail(ORACLE_EINVAL, "tree is not 2:1 balanced");
          int sl = in_face_slot(g, C, axis);
          cn.contrib[s * 4 + sl] = int32_t(k);
        }
        cn.nbr[s] = cn.contrib[s * 4 + 0];
        (void)nsub;
      }
    }
  }
  return 0;
}

// ------------------------------------------------------------------------------------------
// 1D operators (Sec. 2.1): Gauss-Legendre solution points (reading: the paper names no point
// set), Lagrange basis, and the DG correction function g_L = right Radau polynomial of degree
// p+1 (Huynh), g_R(x) = g_L(-x).
// ------------------------------------------------------------------------------------------
void legendre(int n, double x, double& P, double& dP) {
  // three-term recurrence; P'_{k+1} = P'_{k-1} + (2k+1) P_k
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (n == 0) {
    P = 1.0;
    dP = 0.0;
    return;
  }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    double d2 = d0 + (2.0 * k + 1.0) * p1;
    p0 = p1;
    p1 = p2;
    d0 = d1;
    d1 = d2;
  }
  P = p1;
  dP = d1;
}

// Gauss-Legendre nodes by Newton iteration on P_n, weights 2/((1-x^2) P_n'(x)^2); ascending.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n; ++k) {
    double z = std::cos(pi * (k + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(n, z, P, dP);
      double dz = P / dP;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double P, dP;
    legendre(n, z, P, dP);
    x[n - 1 - k] = z;
    w[n - 1 - k] = 2.0 / ((1.0 - z * z) * dP * dP);
  }
}

double lagrange(const std::vector<double>& xs, int j, double x) {
  double r = 1.0;
  for (size_t m = 0; m < xs.size(); ++m)
    if (int(m) != j) r *= (x - xs[m]) / (xs[j] - xs[m]);
  return r;
}

double dlagrange(const std::vector<double>& xs, int j, double x) {
  double s = 0.0;
  for (size_t k = 0; k < xs.size(); ++k) {
    if (int(k) == j) continue;
    double prod = 1.0 / (xs[j] - xs[k]);
    for (size_t m = 0; m < xs.size(); ++m)
      if (int(m) != j && m != k) prod *= (x - xs[m]) / (xs[j] - xs[m]);
    s += prod;
  }
  return s;
}

// g_L = R_{R,p+1} = (-1)^(p+1)/2 (P_{p+1} - P_p); returns g_L'(x).
double dgL(int p, double x) {
  double Pa, dPa, Pb, dPb;
  legendre(p + 1, x, Pa, dPa);
  legendre(p, x, Pb, dPb);
  double sgn = ((p + 1) % 2 == 0) ? 1.0 : -1.0;
  return 0.5 * sgn * (dPa - dPb);
}
double gLval(int p, double x) {
  double Pa, dPa, Pb, dPb;
  legendre(p + 1, x, Pa, dPa);
  legendre(p, x, Pb, dPb);
  double sgn = ((p + 1) % 2 == 0) ? 1.0 : -1.0;
  return 0.5 * sgn * (Pa - Pb);
}

struct Ops1D {
  int p, n;
  std::vector<double> x, w, D, lm, lp, gL, gR;
};

Ops1D make_ops(int p) {
  Ops1D o;
  o.p = p;
  o.n = p + 1;
  gauss_legendre(o.n, o.x, o.w);
  int n = o.n;
  o.D.assign(n * n, 0.0);
  o.lm.assign(n, 0.0);
  o.lp.assign(n, 0.0);
  o.gL.assign(n, 0.0);
  o.gR.assign(n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) o.D[i * n + j] = dlagrange(o.x, j, o.x[i]);
  for (int j = 0; j < n; ++j) {
    o.lm[j] = lagrange(o.x, j, -1.0);
    o.lp[j] = lagrange(o.x, j, 1.0);
  }
  for (int i = 0; i < n; ++i) {
    o.gL[i] = dgL(p, o.x[i]);
    o.gR[i] = -dgL(p, -o.x[i]);  // g_R(x) = g_L(-x)
  }
  return o;
}

// Dense Gaussian elimination with partial pivoting: solves A x = b for several right-hand sides.
void solve_dense(int n, std::vector<double> A, std::vector<double>& B, int nrhs) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (piv != c) {
      for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
      for (int k = 0; k < nrhs; ++k) std::swap(B[c * nrhs + k], B[piv * nrhs + k]);
    }
    for (int r = c + 1; r < n; ++r) {
      double f = A[r * n + c] / A[c * n + c];
      for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      for (int k = 0; k < nrhs; ++k) B[r * nrhs + k] -= f * B[c * nrhs + k];
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    for (int k = 0; k < nrhs; ++k) {
      double s = B[c * nrhs + k];
      for (int j = c + 1; j < n; ++j) s -= A[c * n + j] * B[j * nrhs + k];
      B[c * nrhs + k] = s / A[c * n + c];
    }
  }
}

// Tensor-product Lagrange basis in `dd` dimensions at reference point xi.
double tensor_basis(const std::vector<double>& xs, int dd, int idx, const double* xi) {
  int n = int(xs.size());
  double r = 1.0;
  for (int b = 0; b < dd; ++b) {
    r *= lagrange(xs, idx % n, xi[b]);
    idx /= n;
  }
  return r;
}

// L2 projection operators from 2^dd sub-boxes of [-1,1]^dd onto [-1,1]^dd (Sec. 4.2 restriction
// and Sec. 4.3 mortar back-projection): Mass[j][i] = int l_j l_i over the box, Sub[s][j][i] =
// int over sub-box s of l_j(xi) lhat_i(z(xi)), sub-box s occupying the lower or upper half along
// axis b according to bit b of s (reading: the printed integration domain of S is the sub-box).
// Integrals by a tensor Gauss rule with n+1 points per axis (exact for the degree 2p integrands).
struct Proj {
  int dd, n, Np;
  std::vector<double> mass, sub;  // Np*Np, (2^dd)*Np*Np
};

Proj make_proj(const Ops1D& o, int dd) {
  Proj P;
  P.dd = dd;
  P.n = o.n;
  P.Np = 1;
  for (int b = 0; b < dd; ++b) P.Np *= o.n;
  std::vector<double> qx, qw;
  gauss_legendre(o.n + 1, qx, qw);
  int nq = o.n + 1, Nq = 1;
  for (int b = 0; b < dd; ++b) Nq *= nq;
  int Np = P.Np, nsub = 1 << dd;
  P.mass.assign(Np * Np, 0.0);
  P.sub.assign(nsub * Np * Np, 0.0);
  for (int q = 0; q < Nq; ++q) {
    double z[3] = {0, 0, 0}, wq = 1.0;
    int t = q;
    for (int b = 0; b < dd; ++b) {
      z[b] = qx[t % nq];
      wq *= qw[t % nq];
      t /= nq;
    }
    for (int j = 0; j < Np; ++j)
      for (int i = 0; i < Np; ++i)
        P.mass[j * Np + i] += wq * tensor_basis(o.x, dd, j, z) * tensor_basis(o.x, dd, i, z);
    for (int s = 0; s < nsub; ++s) {
      double xi[3] = {0, 0, 0};
      for (int b = 0; b < dd; ++b) xi[b] = (z[b] + 2.0 * ((s >> b) & 1) - 1.0) / 2.0;
      double jac = std::pow(0.5, dd);  // d xi = 2^-dd d z
      for (int j = 0; j < Np; ++j)
        for (int i = 0; i < Np; ++i)
          P.sub[(s * Np + j) * Np + i] +=
              wq * jac * tensor_basis(o.x, dd, j, xi) * tensor_basis(o.x, dd, i, z);
    }
  }
  return P;
}

// u_out = Mass^{-1} sum_s Sub[s] u_s for `nv` fields; in holds [2^dd][nv][Np], out [nv][Np].
void apply_proj(const Proj& P, int nv, const double* in, double* out) {
  int Np = P.Np, nsub = 1 << P.dd;
  std::vector<double> rhs(Np * nv, 0.0);
  for (int s = 0; s < nsub; ++s)
    for (int v = 0; v < nv; ++v)
      for (int j = 0; j < Np; ++j)
        for (int i = 0; i < Np; ++i)
          rhs[j * nv + v] += P.sub[(s * Np + j) * Np + i] * in[(s * nv + v) * Np + i];
  solve_dense(Np, P.mass, rhs, nv);
  for (int v = 0; v < nv; ++v)
    for (int j = 0; j < Np; ++j) out[v * Np + j] = rhs[j * nv + v];
}

// ------------------------------------------------------------------------------------------
// Euler equations, Rusanov flux (Sec. 4.3) and the isentropic vortex (Sec. 5.2)
// ------------------------------------------------------------------------------------------
void euler_flux(int dim, double gamma, const double* q, int a, double* f) {
  double rho = q[0], vel[3] = {0, 0, 0}, ke = 0.0;
  for (int b = 0; b < dim; ++b) {
    vel[b] = q[1 + b] / rho;
    ke += 0.5 * rho * vel[b] * vel[b];
  }
  double E = q[1 + dim];
  double p = (gamma - 1.0) * (E - ke);
  f[0] = q[1 + a];
  for (int b = 0; b < dim; ++b) f[1 + b] = q[1 + b] * vel[a] + (b == a ? p : 0.0);
  f[1 + dim] = (E + p) * vel[a];
}

double wave_speed(int dim, double gamma, const double* q, int a) {
  double rho = q[0], ke = 0.0;
  for (int b = 0; b < dim; ++b) ke += 0.5 * q[1 + b] * q[1 + b] / rho;
  double p = (gamma - 1.0) * (q[1 + dim] - ke);
  double c = std::sqrt(gamma * p / rho);
  return std::fabs(q[1 + a] / rho) + c;
}

// Rusanov common flux along +axis between the minus-side state qL and the plus-side state qR.
// Reading: lambda = max(|u_n|+c) of the two states, pointwise.
void rusanov(int dim, double gamma, const double* qL, const double* qR, int a, double* F) {
  int nv = dim + 2;
  double fL[5], fR[5];
  euler_flux(dim, gamma, qL, a, fL);
  euler_flux(dim, gamma, qR, a, fR);
  double lam = std::max(wave_speed(dim, gamma, qL, a), wave_speed(dim, gamma, qR, a));
  for (int v = 0; v < nv; ++v) F[v] = 0.5 * (fL[v] + fR[v]) - 0.5 * lam * (qR[v] - qL[v]);
}

struct Cfg {
  int dim, p;
  double L;
  int Dbase, Dmax;
  double gamma;
  std::vector<std::array<double, 4>> vort;
  double uinf[3], rho_inf, p_inf, cfl, dt;
  int adapt_every, indicator;
  double th_refine, th_coarsen;
  int init_passes;
};

// Advected isentropic vortex (Sec. 5.2).  Reading: r is the distance to the vortex axis scaled by
// the core radius, the exponent uses r^2 with phi = 1/2, beta plays alpha, T = p/rho, and the
// state is isentropic: rho = rho_inf (T/T_inf)^(1/(gamma-1)), p = rho T.  Several vortices add
// their perturbations; each centre moves with the freestream and the nearest periodic image is used.
void exact_state(const Cfg& c, double t, const double* X, double* q) {
  const double pi = 3.14159265358979323846;
  double du = 0.0, dv = 0.0, dT = 0.0;
  for (const auto& v : c.vort) {
    double cx = v[0] + c.uinf[0] * t, cy = v[1] + c.uinf[1] * t;
    double dx = X[0] - cx, dy = X[1] - cy;
    dx -= c.L * std::floor(dx / c.L + 0.5);
    dy -= c.L * std::floor(dy / c.L + 0.5);
    double beta = v[2], R = v[3];
    double r2 = (dx * dx + dy * dy) / (R * R);
    double e = std::exp(0.5 * (1.0 - r2));
    du += -beta / (2.0 * pi) * (dy / R) * e;
    dv += beta / (2.0 * pi) * (dx / R) * e;
    dT += -(c.gamma - 1.0) * beta * beta / (8.0 * c.gamma * pi * pi) * std::exp(1.0 - r2);
  }
  double Tinf = c.p_inf / c.rho_inf;
  double T = Tinf + dT;
  double rho = c.rho_inf * std::pow(T / Tinf, 1.0 / (c.gamma - 1.0));
  double p = rho * T;
  double vel[3] = {c.uinf[0] + du, c.uinf[1] + dv, c.uinf[2]};
  q[0] = rho;
  double ke = 0.0;
  for (int b = 0; b < c.dim; ++b) {
    q[1 + b] = rho * vel[b];
    ke += 0.5 * rho * vel[b] * vel[b];
  }
  q[1 + c.dim] = p / (c.gamma - 1.0) + ke;
}

// ------------------------------------------------------------------------------------------
// Mesh state and the FR residual (Sec. 2.1 corrected-flux derivative, Sec. 4.3 common fluxes)
// ------------------------------------------------------------------------------------------
struct MeshO {
  Cfg c;
  Geo g;
  Ops1D o;
  Proj face_proj, vol_proj;
  int n, N, Nf, nv, nf;
  std::vector<uint64_t> keys;
  std::vector<double> u;
  Conn conn;
  double t = 0.0, dt = 0.0;
  int64_t step = 0;
};

int pidx(int n, const int* i) { return i[0] + n * (i[1] + n * i[2]); }

// Element point indices of face point q on the face of `axis` at line position j along the axis.
void face_line_point(int dim, int n, int axis, int q, int j, int* i) {
  i[0] = i[1] = i[2] = 0;
  int t = q;
  for (int b = 0; b < dim; ++b) {
    if (b == axis) continue;
    i[b] = t % n;
    t /= n;
  }
  i[axis] = j;
}

double elem_h(const MeshO& m, int64_t e) {
  Box b = decode(m.g, m.keys[e]);
  return m.c.L / double(int64_t(1) << b.depth);
}

void point_coords(const MeshO& m, int64_t e, const int* i, double* X) {
  Box b = decode(m.g, m.keys[e]);
  double h = elem_h(m, e);
  double fine = m.c.L / double(int64_t(1) << m.g.Dmax);
  for (int a = 0; a < 3; ++a) X[a] = 0.0;
  for (int a = 0; a < m.c.dim; ++a) X[a] = b.x[a] * fine + 0.5 * h * (m.o.x[i[a]] + 1.0);
}

// R(u) for the whole mesh; u and R are [M][nv][N].
void residual(const MeshO& m, const std::vector<double>& u, std::vector<double>& R) {
  int dim = m.c.dim, n = m.n, N = m.N, Nf = m.Nf, nv = m.nv, nf = m.nf;
  size_t M = m.keys.size();
  double gam = m.c.gamma;
  const Ops1D& o = m.o;
  // 1. solution -> flux points: face traces tr[e][f][v][q] (mortar algorithm, step 1)
  std::vector<double> tr(M * nf * nv * Nf, 0.0);
  for (size_t e = 0; e < M; ++e)
    for (int f = 0; f < nf; ++f) {
      int axis = f / 2;
      const std::vector<double>& lf = (f % 2) ? o.lp : o.lm;
      for (int v = 0; v < nv; ++v)
        for (int q = 0; q < Nf; ++q) {
          double s = 0.0;
          for (int j = 0; j < n; ++j) {
            int i[3];
            face_line_point(dim, n, axis, q, j, i);
            s += lf[j] * u[(e * nv + v) * N + pidx(n, i)];
          }
          tr[((e * nf + f) * nv + v) * Nf + q] = s;
        }
    }
  auto trace = [&](size_t e, int f, int q, double* qv) {
    for (int v = 0; v < nv; ++v) qv[v] = tr[((e * nf + f) * nv + v) * Nf + q];
  };
  // 2. common fluxes Fc[e][f][v][q] along +axis
  std::vector<double> Fc(M * nf * nv * Nf, 0.0);
  // 2a. conforming faces and the fine sides of hanging faces (mortar steps 2-3: the coarse
  //     trace polynomial is projected, i.e. interpolated, onto the mortar piece)
  for (size_t e = 0; e < M; ++e)
    for (int f = 0; f < nf; ++f) {
      size_t s = e * nf + f;
      int axis = f / 2, side = f % 2;
      if (m.conn.ftype[s] == 2) continue;
      size_t nb = size_t(m.conn.nbr[s]);
      for (int q = 0; q < Nf; ++q) {
        double qo[5], qn[5], F[5];
        trace(e, f, q, qo);
        if (m.conn.ftype[s] == 0) {
          trace(nb, f ^ 1, q, qn);
        } else {
          // point q of this (fine) face in the coarse face's reference coordinates
          Box K = decode(m.g, m.keys[e]);
          int cidx = child_index(m.g, K);
          double eta[2] = {0, 0};
          int t = q, fb = 0;
          for (int b = 0; b < dim; ++b) {
            if (b == axis) continue;
            double xi = o.x[t % n];
            t /= n;
            eta[fb++] = (xi + 2.0 * ((cidx >> b) & 1) - 1.0) / 2.0;
          }
          for (int v = 0; v < nv; ++v) {
            double sacc = 0.0;
            for (int q2 = 0; q2 < Nf; ++q2)
              sacc += tensor_basis(o.x, dim - 1, q2, eta) * tr[((nb * nf + (f ^ 1)) * nv + v) * Nf + q2];
            qn[v] = sacc;
          }
        }
        if (side == 0)
          rusanov(dim, gam, qn, qo, axis, F);
        else
          rusanov(dim, gam, qo, qn, axis, F);
        for (int v = 0; v < nv; ++v) Fc[(s * nv + v) * Nf + q] = F[v];
      }
    }
  // 2b. coarse sides of hanging faces: L2 projection of the mortar fluxes (mortar step 4)
  for (size_t e = 0; e < M; ++e)
    for (int f = 0; f < nf; ++f) {
      size_t s = e * nf + f;
      if (m.conn.ftype[s] != 2) continue;
      int nsub = 1 << (dim - 1);
      std::vector<double> in(nsub * nv * Nf), out(nv * Nf);
      for (int sl = 0; sl < nsub; ++sl) {
        size_t k = size_t(m.conn.contrib[s * 4 + sl]);
        for (int v = 0; v < nv; ++v)
          for (int q = 0; q < Nf; ++q)
            in[(sl * nv + v) * Nf + q] = Fc[((k * nf + (f ^ 1)) * nv + v) * Nf + q];
      }
      apply_proj(m.face_proj, nv, in.data(), out.data());
      for (int v = 0; v < nv; ++v)
        for (int q = 0; q < Nf; ++q) Fc[(s * nv + v) * Nf + q] = out[v * Nf + q];
    }
  // 3. corrected flux derivative per axis and line (Sec. 2.1), R = -sum_a (2/h) dfhat_a/dxi
  R.assign(M * nv * N, 0.0);
  for (size_t e = 0; e < M; ++e) {
    double h = elem_h(m, e);
    for (int axis = 0; axis < dim; ++axis)
      for (int q = 0; q < Nf; ++q) {
        // flux at the n points of the line
        std::vector<double> fl(n * nv);
        for (int j = 0; j < n; ++j) {
          int i[3];
          face_line_point(dim, n, axis, q, j, i);
          double qv[5];
          for (int v = 0; v < nv; ++v) qv[v] = u[(e * nv + v) * N + pidx(n, i)];
          euler_flux(dim, gam, qv, axis, &fl[j * nv]);
        }
        for (int v = 0; v < nv; ++v) {
          double fm = 0.0, fp = 0.0;  // discontinuous flux polynomial at xi = -1, +1
          for (int j = 0; j < n; ++j) {
            fm += o.lm[j] * fl[j * nv + v];
            fp += o.lp[j] * fl[j * nv + v];
          }
          double Fm = Fc[((e * nf + 2 * axis) * nv + v) * Nf + q];
          double Fp = Fc[((e * nf + 2 * axis + 1) * nv + v) * Nf + q];
          for (int ii = 0; ii < n; ++ii) {
            double d = 0.0;
            for (int j = 0; j < n; ++j) d += o.D[ii * n + j] * fl[j * nv + v];
            d += o.gL[ii] * (Fm - fm) + o.gR[ii] * (Fp - fp);
            int i[3];
            face_line_point(dim, n, axis, q, ii, i);
            R[(e * nv + v) * N + pidx(n, i)] -= (2.0 / h) * d;
          }
        }
      }
  }
}

// SSP-RK3 (Eq. rk3) with a fixed dt.
void rk3_step(MeshO& m) {
  std::vector<double> R, u1, u2;
  const std::vector<double>& un = m.u;
  size_t S = un.size();
  residual(m, un, R);
  u1.resize(S);
  for (size_t k = 0; k < S; ++k) u1[k] = un[k] + m.dt * R[k];
  residual(m, u1, R);
  u2.resize(S);
  for (size_t k = 0; k < S; ++k) u2[k] = 0.75 * un[k] + 0.25 * u1[k] + 0.25 * m.dt * R[k];
  residual(m, u2, R);
  std::vector<double> u3(S);
  for (size_t k = 0; k < S; ++k)
    u3[k] = (1.0 / 3.0) * un[k] + (2.0 / 3.0) * u2[k] + (2.0 / 3.0) * m.dt * R[k];
  m.u.swap(u3);
  m.t += m.dt;
  m.step += 1;
}

void set_ic(MeshO& m, double t) {
  size_t M = m.keys.size();
  m.u.assign(M * m.nv * m.N, 0.0);
  for (size_t e = 0; e < M; ++e)
    for (int pt = 0; pt < m.N; ++pt) {
      int i[3] = {pt % m.n, (pt / m.n) % m.n, m.c.dim == 3 ? pt / (m.n * m.n) : 0};
      double X[3], q[5];
      point_coords(m, int64_t(e), i, X);
      exact_state(m.c, t, X, q);
      for (int v = 0; v < m.nv; ++v) m.u[(e * m.nv + v) * m.N + pt] = q[v];
    }
}

// Adaptation indicators.  Reading (density gradient, not in the paper): eta = h * max_i |grad rho|
// with the uncorrected local derivative (2/h) sum_j l_j' rho_j; refine above th_refine, coarsen
// below th_coarsen.  Analytic centre (Sec. 5.2): compare the numbers of solution points closer
// than th_refine and farther than th_coarsen from the nearest vortex axis.
void indicator_flags(const MeshO& m, std::vector<int8_t>& flags, std::vector<double>& eta) {
  size_t M = m.keys.size();
  int n = m.n, N = m.N, dim = m.c.dim;
  flags.assign(M, 0);
  eta.assign(M, 0.0);
  for (size_t e = 0; e < M; ++e) {
    double h = elem_h(m, int64_t(e));
    if (m.c.indicator == 0) {
      double gmax = 0.0;
      for (int pt = 0; pt < N; ++pt) {
        int i[3] = {pt % n, (pt / n) % n, dim == 3 ? pt / (n * n) : 0};
        double g2 = 0.0;
        for (int a = 0; a < dim; ++a) {
          double d = 0.0;
          for (int j = 0; j < n; ++j) {
            int k[3] = {i[0], i[1], i[2]};
            k[a] = j;
            d += m.o.D[i[a] * n + j] * m.u[(e * m.nv + 0) * N + pidx(n, k)];
          }
          d *= 2.0 / h;
          g2 += d * d;
        }
        gmax = std::max(gmax, std::sqrt(g2));
      }
      eta[e] = h * gmax;
      flags[e] = eta[e] > m.c.th_refine ? 1 : (eta[e] < m.c.th_coarsen ? -1 : 0);
    } else if (m.c.indicator == 1) {
      int nin = 0, nout = 0;
      for (int pt = 0; pt < N; ++pt) {
        int i[3] = {pt % n, (pt / n) % n, dim == 3 ? pt / (n * n) : 0};
        double X[3];
        point_coords(m, int64_t(e), i, X);
        double rmin = 1e300;
        for (const auto& v : m.c.vort) {
          double dx = X[0] - (v[0] + m.c.uinf[0] * m.t), dy = X[1] - (v[1] + m.c.uinf[1] * m.t);
          dx -= m.c.L * std::floor(dx / m.c.L + 0.5);
          dy -= m.c.L * std::floor(dy / m.c.L + 0.5);
          rmin = std::min(rmin, std::sqrt(dx * dx + dy * dy));
        }
        if (rmin < m.c.th_refine) ++nin;
        if (rmin > m.c.th_coarsen) ++nout;
      }
      eta[e] = double(nin - nout);
      flags[e] = nin > nout ? 1 : (nin < nout ? -1 : 0);
    }
  }
}

// Solution transfer (Sec. 4.2): copy, interpolation of the parent polynomial at the child points
// (Eq. parent_soln), or L2 projection of the fused children onto the parent.
void transfer(MeshO& m, const std::vector<uint64_t>& old_keys, const std::vector<double>& uo,
              const std::vector<uint64_t>& new_keys, std::vector<double>& un) {
  std::vector<int32_t> src;
  std::vector<int8_t> tag;
  map_trees(m.g, old_keys, new_keys, src, tag);
  int n = m.n, N = m.N, nv = m.nv, dim = m.c.dim;
  size_t E = size_t(N) * nv;
  un.assign(new_keys.size() * E, 0.0);
  for (size_t j = 0; j < new_keys.size(); ++j) {
    size_t i = size_t(src[j]);
    if (tag[j] == 0) {
      for (size_t k = 0; k < E; ++k) un[j * E + k] = uo[i * E + k];
    } else if (tag[j] == 1) {
      Box A = decode(m.g, old_keys[i]), K = decode(m.g, new_keys[j]);
      double wA = double(width(m.g, A.depth)), wK = double(width(m.g, K.depth));
      for (int pt = 0; pt < N; ++pt) {
        int ii[3] = {pt % n, (pt / n) % n, dim == 3 ? pt / (n * n) : 0};
        double xi[3] = {0, 0, 0};
        for (int a = 0; a < dim; ++a)
          xi[a] = -1.0 + 2.0 * (double(K.x[a] - A.x[a]) + 0.5 * (m.o.x[ii[a]] + 1.0) * wK) / wA;
        for (int v = 0; v < nv; ++v) {
          double s = 0.0;
          for (int q = 0; q < N; ++q) s += tensor_basis(m.o.x, dim, q, xi) * uo[i * E + v * N + q];
          un[j * E + v * N + pt] = s;
        }
      }
    } else {
      // children i .. i+2^dim-1 in Morton order = child index order
      apply_proj(m.vol_proj, nv, &uo[i * E], &un[j * E]);
    }
  }
}

int mesh_from_cfg(const oracle_config* in, MeshO& m) {
  if (!in) return fail(ORACLE_EINVAL, "null config");
  Cfg& c = m.c;
  c.dim = in->dim;
  c.p = in->p;
  c.L = in->L;
  c.Dbase = in->Dbase;
  c.Dmax = in->Dmax;
  c.gamma = in->gamma;
  c.vort.clear();
  for (int k = 0; k < in->nvort; ++k)
    c.vort.push_back({in->vort[4 * k], in->vort[4 * k + 1], in->vort[4 * k + 2], in->vort[4 * k + 3]});
  for (int a = 0; a < 3; ++a) c.uinf[a] = in->uinf[a];
  c.rho_inf = in->rho_inf;
  c.p_inf = in->p_inf;
  c.cfl = in->cfl;
  c.dt = in->dt;
  c.adapt_every = in->adapt_every;
  c.indicator = in->indicator;
  c.th_refine = in->th_refine;
  c.th_coarsen = in->th_coarsen;
  c.init_passes = in->init_passes;
  if (!geo_ok(c.dim, c.Dmax)) return fail(ORACLE_EINVAL, "dim/Dmax out of range");
  if (c.p < 1 || c.p > 4) return fail(ORACLE_EINVAL, "p out of range");
  if (c.Dbase < 1 || c.Dbase > c.Dmax) return fail(ORACLE_EINVAL, "Dbase out of range");
  if (!(c.L > 0) || !(c.gamma > 1)) return fail(ORACLE_EINVAL, "bad L or gamma");
  m.g = Geo{c.dim, c.Dmax, depth_bits(c.Dmax)};
  m.o = make_ops(c.p);
  m.n = c.p + 1;
  m.N = c.dim == 2 ? m.n * m.n : m.n * m.n * m.n;
  m.Nf = c.dim == 2 ? m.n : m.n * m.n;
  m.nv = c.dim + 2;
  m.nf = 2 * c.dim;
  m.face_proj = make_proj(m.o, c.dim - 1);
  m.vol_proj = make_proj(m.o, c.dim);
  return 0;
}

int do_adapt(MeshO& m, const int8_t* flags, bool transfer_state) {
  std::vector<uint64_t> nk = adapt_keys(m.g, m.c.Dbase, m.keys, flags);
  if (transfer_state) {
    std::vector<double> un;
    transfer(m, m.keys, m.u, nk, un);
    m.u.swap(un);
  }
  m.keys.swap(nk);
  return build_conn(m.g, m.keys, m.conn);
}

}  // namespace

struct oracle_mesh {
  MeshO m;
};

extern "C" {

const char* oracle_last_error(void) { return g_err.c_str(); }

int oracle_morton_encode(int dim, int Dmax, int64_t n, const int32_t* boxes, uint64_t* keys) {
  if (!geo_ok(dim, Dmax) || n < 0) return fail(ORACLE_EINVAL, "bad geometry");
  Geo g{dim, Dmax, depth_bits(Dmax)};
  for (int64_t k = 0; k < n; ++k) {
    Box b{};
    b.depth = boxes[4 * k];
    for (int a = 0; a < 3; ++a) b.x[a] = boxes[4 * k + 1 + a];
    if (b.depth < 0 || b.depth > Dmax) return fail(ORACLE_EINVAL, "depth out of range");
    keys[k] = encode(g, b);
  }
  return 0;
}

int oracle_morton_decode(int dim, int Dmax, int64_t n, const uint64_t* keys, int32_t* boxes) {
  if (!geo_ok(dim, Dmax) || n < 0) return fail(ORACLE_EINVAL, "bad geometry");
  Geo g{dim, Dmax, depth_bits(Dmax)};
  for (int64_t k = 0; k < n; ++k) {
    Box b = decode(g, keys[k]);
    boxes[4 * k] = b.depth;
    for (int a = 0; a < 3; ++a) boxes[4 * k + 1 + a] = int32_t(b.x[a]);
  }
  return 0;
}

int oracle_linearise(int dim, int Dmax, const uint64_t* keys, int64_t n, uint64_t* out,
                     int64_t cap, int64_t* n_out) {
  if (!geo_ok(dim, Dmax) || n < 0) return fail(ORACLE_EINVAL, "bad geometry");
  Geo g{dim, Dmax, depth_bits(Dmax)};
  std::vector<uint64_t> r = linearise(g, std::vector<uint64_t>(keys, keys + n));
  *n_out = int64_t(r.size());
  if (int64_t(r.size()) > cap) return fail(ORACLE_EOVERFLOW, "output capacity too small");
  std::copy(r.begin(), r.end(), out);
  return 0;
}

int oracle_tree_complete(int dim, int Dmin, int Dmax, double L, const double* pts, int64_t n,
                         uint64_t* out, int64_t cap, int64_t* n_out) {
  if (!geo_ok(dim, Dmax) || Dmin < 0 || Dmin > Dmax || !(L > 0) || n < 0)
    return fail(ORACLE_EINVAL, "bad arguments");
  Geo g{dim, Dmax, depth_bits(Dmax)};
  int64_t side = int64_t(1) << Dmax;
  std::set<uint64_t> cells;
  for (int64_t k = 0; k < n; ++k) {
    Box b{};
    b.depth = Dmax;
    for (int a = 0; a < dim; ++a) {
      double c = std::floor(pts[k * dim + a] / L * double(side));
      int64_t ci = c < 0 ? 0 : (c >= double(side) ? side - 1 : int64_t(c));
      b.x[a] = ci;
    }
    cells.insert(encode(g, b));
  }
  std::vector<uint64_t> r;
  Box root{};
  root.depth = 0;
  complete_rec(g, Dmin, cells, root, r);
  *n_out = int64_t(r.size());
  if (int64_t(r.size()) > cap) return fail(ORACLE_EOVERFLOW, "output capacity too small");
  std::copy(r.begin(), r.end(), out);
  return 0;
}

int oracle_balance(int dim, int Dmax, const uint64_t* keys, int64_t n, uint64_t* out, int64_t cap,
                   int64_t* n_out) {
  if (!geo_ok(dim, Dmax) || n < 0) return fail(ORACLE_EINVAL, "bad geometry");
  Geo g{dim, Dmax, depth_bits(Dmax)};
  std::vector<uint64_t> in(keys, keys + n);
  if (!complete(g, in)) return fail(ORACLE_EINVAL, "input is not a complete linear tree");
  std::vector<uint64_t> r = balance(g, in);
  *n_out = int64_t(r.size());
  if (int64_t(r.size()) > cap) return fail(ORACLE_EOVERFLOW, "output capacity too small");
  std::copy(r.begin(), r.end(), out);
  return 0;
}

int oracle_adapt_keys(int dim, int Dbase, int Dmax, const uint64_t* keys, const int8_t* flags,
                      int64_t n, uint64_t* out, int64_t cap, int64_t* n_out) {
  if (!geo_ok(dim, Dmax) || n < 0) return fail(ORACLE_EINVAL, "bad geometry");
  Geo g{dim, Dmax, depth_bits(Dmax)};
  std::vector<uint64_t> in(keys, keys + n);
  if (!complete(g, in)) return fail(ORACLE_EINVAL, "input is not a complete linear tree");
  std::vector<uint64_t> r = adapt_keys(g, Dbase, in, flags);
  *n_out = int64_t(r.size());
  if (int64_t(r.size()) > cap) return fail(ORACLE_EOVERFLOW, "output capacity too small");
  std::copy(r.begin(), r.end(), out);
  return 0;
}

int oracle_map(int dim, int Dmax, const uint64_t* old_keys, int64_t n_old, const uint64_t* new_keys,
               int64_t n_new, int32_t* src, int8_t* tag) {
  if (!geo_ok(dim, Dmax)) return fail(ORACLE_EINVAL, "bad geometry");
  Geo g{dim, Dmax, depth_bits(Dmax)};
  std::vector<uint64_t> o(old_keys, old_keys + n_old), nn(new_keys, new_keys + n_new);
  if (!complete(g, o) || !complete(g, nn)) return fail(ORACLE_EINVAL, "inputs must be complete");
  std::vector<int32_t> s;
  std::vector<int8_t> t;
  map_trees(g, o, nn, s, t);
  std::copy(s.begin(), s.end(), src);
  std::copy(t.begin(), t.end(), tag);
  return 0;
}

int oracle_conn(int dim, int Dmax, const uint64_t* keys, int64_t n, int32_t* nbr, int8_t* ftype,
                int8_t* slot) {
  if (!geo_ok(dim, Dmax)) return fail(ORACLE_EINVAL, "bad geometry");
  Geo g{dim, Dmax, depth_bits(Dmax)};
  std::vector<uint64_t> k(keys, keys + n);
  if (!complete(g, k)) return fail(ORACLE_EINVAL, "input is not a complete linear tree");
  Conn cn;
  int rc = build_conn(g, k, cn);
  if (rc) return rc;
  std::copy(cn.nbr.begin(), cn.nbr.end(), nbr);
  std::copy(cn.ftype.begin(), cn.ftype.end(), ftype);
  std::copy(cn.slot.begin(), cn.slot.end(), slot);
  return 0;
}

int oracle_operators(int p, double* x, double* w, double* D, double* lm, double* lp, double* gL,
                     double* gR) {
  if (p < 1 || p > 8) return fail(ORACLE_EINVAL, "p out of range");
  Ops1D o = make_ops(p);
  std::copy(o.x.begin(), o.x.end(), x);
  std::copy(o.w.begin(), o.w.end(), w);
  std::copy(o.D.begin(), o.D.end(), D);
  std::copy(o.lm.begin(), o.lm.end(), lm);
  std::copy(o.lp.begin(), o.lp.end(), lp);
  std::copy(o.gL.begin(), o.gL.end(), gL);
  std::copy(o.gR.begin(), o.gR.end(), gR);
  return 0;
}

double oracle_correction_gL(int p, double x) { return gLval(p, x); }

double oracle_rk3_scalar(double lam, double u0, double dt) {
  // Eq. rk3 with R(u) = lam*u
  double u1 = u0 + dt * lam * u0;
  double u2 = 0.75 * u0 + 0.25 * u1 + 0.25 * dt * lam * u1;
  return (1.0 / 3.0) * u0 + (2.0 / 3.0) * u2 + (2.0 / 3.0) * dt * lam * u2;
}

int oracle_prolong(int dim, int p, int nv, const double* parent, int child, double* out) {
  if ((dim != 2 && dim != 3) || p < 1 || p > 8) return fail(ORACLE_EINVAL, "bad args");
  Ops1D o = make_ops(p);
  int n = p + 1, N = dim == 2 ? n * n : n * n * n;
  for (int pt = 0; pt < N; ++pt) {
    int ii[3] = {pt % n, (pt / n) % n, dim == 3 ? pt / (n * n) : 0};
    double xi[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) xi[a] = (o.x[ii[a]] + 2.0 * ((child >> a) & 1) - 1.0) / 2.0;
    for (int v = 0; v < nv; ++v) {
      double s = 0.0;
      for (int q = 0; q < N; ++q) s += tensor_basis(o.x, dim, q, xi) * parent[v * N + q];
      out[v * N + pt] = s;
    }
  }
  return 0;
}

int oracle_restrict(int dim, int p, int nv, const double* children, double* out) {
  if ((dim != 2 && dim != 3) || p < 1 || p > 8) return fail(ORACLE_EINVAL, "bad args");
  Ops1D o = make_ops(p);
  Proj P = make_proj(o, dim);
  apply_proj(P, nv, children, out);
  return 0;
}

int oracle_exact(const oracle_config* cfg, double t, int64_t npts, const double* xyz, double* q) {
  MeshO m;
  int rc = mesh_from_cfg(cfg, m);
  if (rc) return rc;
  for (int64_t k = 0; k < npts; ++k) exact_state(m.c, t, &xyz[3 * k], &q[k * m.nv]);
  return 0;
}

int oracle_mesh_init(const oracle_config* cfg, oracle_mesh** out) {
  auto* h = new oracle_mesh();
  MeshO& m = h->m;
  int rc = mesh_from_cfg(cfg, m);
  if (rc) {
    delete h;
    return rc;
  }
  // Reading of the initial mesh: uniform at Dbase, then passes of {closed-form state, flags,
  // adaptation} with the state re-evaluated from the closed form after each pass.
  int64_t side = int64_t(1) << m.c.Dbase;
  int64_t cnt = m.c.dim == 2 ? side * side : side * side * side;
  m.keys.clear();
  for (int64_t k = 0; k < cnt; ++k) {
    Box b{};
    b.depth = m.c.Dbase;
    b.x[0] = (k % side) * width(m.g, m.c.Dbase);
    b.x[1] = ((k / side) % side) * width(m.g, m.c.Dbase);
    b.x[2] = m.c.dim == 3 ? (k / (side * side)) * width(m.g, m.c.Dbase) : 0;
    m.keys.push_back(encode(m.g, b));
  }
  std::sort(m.keys.begin(), m.keys.end());
  int passes = m.c.init_passes < 0 ? m.c.Dmax - m.c.Dbase : m.c.init_passes;
  for (int ps = 0; ps < passes; ++ps) {
    set_ic(m, 0.0);
    std::vector<int8_t> fl;
    std::vector<double> eta;
    indicator_flags(m, fl, eta);
    m.keys = adapt_keys(m.g, m.c.Dbase, m.keys, fl.data());
  }
  set_ic(m, 0.0);
  rc = build_conn(m.g, m.keys, m.conn);
  if (rc) {
    delete h;
    return rc;
  }
  // Reading of the time step: dt = CFL h(Dmax) / ((2p+1) max(|v|+c)) over the initial state.
  if (m.c.dt > 0) {
    m.dt = m.c.dt;
  } else {
    double smax = 0.0;
    for (size_t e = 0; e < m.keys.size(); ++e)
      for (int pt = 0; pt < m.N; ++pt) {
        double q[5];
        for (int v = 0; v < m.nv; ++v) q[v] = m.u[(e * m.nv + v) * m.N + pt];
        double speed2 = 0.0;
        for (int b = 0; b < m.c.dim; ++b) speed2 += (q[1 + b] / q[0]) * (q[1 + b] / q[0]);
        double ke = 0.5 * q[0] * speed2;
        double p = (m.c.gamma - 1.0) * (q[1 + m.c.dim] - ke);
        smax = std::max(smax, std::sqrt(speed2) + std::sqrt(m.c.gamma * p / q[0]));
      }
    double hmin = m.c.L / double(int64_t(1) << m.c.Dmax);
    m.dt = m.c.cfl * hmin / ((2.0 * m.c.p + 1.0) * smax);
  }
  *out = h;
  return 0;
}

void oracle_mesh_free(oracle_mesh* h) { delete h; }

int oracle_step(oracle_mesh* h, int nsteps) {
  if (!h || nsteps < 0) return fail(ORACLE_EINVAL, "bad args");
  for (int s = 0; s < nsteps; ++s) rk3_step(h->m);
  return 0;
}

int oracle_run(oracle_mesh* h, int nsteps) {
  if (!h || nsteps < 0) return fail(ORACLE_EINVAL, "bad args");
  for (int s = 0; s < nsteps; ++s) {
    rk3_step(h->m);
    if (h->m.c.adapt_every > 0 && h->m.step % h->m.c.adapt_every == 0) {
      int rc = oracle_adapt(h, nullptr);
      if (rc) return rc;
    }
  }
  return 0;
}

int oracle_adapt(oracle_mesh* h, const int8_t* flags_or_null) {
  if (!h) return fail(ORACLE_EINVAL, "null mesh");
  MeshO& m = h->m;
  std::vector<int8_t> fl;
  if (flags_or_null) {
    fl.assign(flags_or_null, flags_or_null + m.keys.size());
  } else if (m.c.indicator == 2) {
    fl.assign(m.keys.size(), 0);
  } else {
    std::vector<double> eta;
    indicator_flags(m, fl, eta);
  }
  return do_adapt(m, fl.data(), true);
}

int oracle_flags(oracle_mesh* h, int8_t* flags, double* eta_or_null, int64_t cap) {
  if (!h) return fail(ORACLE_EINVAL, "null mesh");
  if (cap < int64_t(h->m.keys.size())) return fail(ORACLE_EOVERFLOW, "capacity");
  std::vector<int8_t> fl;
  std::vector<double> eta;
  indicator_flags(h->m, fl, eta);
  std::copy(fl.begin(), fl.end(), flags);
  if (eta_or_null) std::copy(eta.begin(), eta.end(), eta_or_null);
  return 0;
}

int oracle_rhs(oracle_mesh* h, double* R, int64_t cap) {
  if (!h) return fail(ORACLE_EINVAL, "null mesh");
  if (cap < int64_t(h->m.u.size())) return fail(ORACLE_EOVERFLOW, "capacity");
  std::vector<double> r;
  residual(h->m, h->m.u, r);
  std::copy(r.begin(), r.end(), R);
  return 0;
}

// L2 norm of the density error (Sec. 5.2) and conserved integrals, by Gauss quadrature at the
// solution points times the element Jacobian (h/2)^dim (reading: the paper names no rule).
int oracle_norms(oracle_mesh* h, oracle_norms_out* out) {
  if (!h || !out) return fail(ORACLE_EINVAL, "null argument");
  MeshO& m = h->m;
  double err = 0.0, integ[5] = {0, 0, 0, 0, 0}, rmin = 1e300, pmin = 1e300;
  for (size_t e = 0; e < m.keys.size(); ++e) {
    double J = std::pow(elem_h(m, int64_t(e)) / 2.0, m.c.dim);
    for (int pt = 0; pt < m.N; ++pt) {
      int i[3] = {pt % m.n, (pt / m.n) % m.n, m.c.dim == 3 ? pt / (m.n * m.n) : 0};
      double W = 1.0;
      for (int a = 0; a < m.c.dim; ++a) W *= m.o.w[i[a]];
      double X[3], qe[5], q[5] = {0, 0, 0, 0, 0};
      point_coords(m, int64_t(e), i, X);
      exact_state(m.c, m.t, X, qe);
      for (int v = 0; v < m.nv; ++v) q[v] = m.u[(e * m.nv + v) * m.N + pt];
      err += W * J * (qe[0] - q[0]) * (qe[0] - q[0]);
      for (int v = 0; v < m.nv; ++v) integ[v] += W * J * q[v];
      double ke = 0.0;
      for (int b = 0; b < m.c.dim; ++b) ke += 0.5 * q[1 + b] * q[1 + b] / q[0];
      double p = (m.c.gamma - 1.0) * (q[1 + m.c.dim] - ke);
      rmin = std::min(rmin, q[0]);
      pmin = std::min(pmin, p);
    }
  }
  out->t = m.t;
  out->l2_rho = std::sqrt(err);
  for (int v = 0; v < 5; ++v) out->integral[v] = v < m.nv ? integ[v] : 0.0;
  out->min_rho = rmin;
  out->min_p = pmin;
  out->M = int64_t(m.keys.size());
  return 0;
}

int oracle_get_leaves(oracle_mesh* h, uint64_t* keys, int64_t cap, int64_t* M) {
  if (!h) return fail(ORACLE_EINVAL, "null mesh");
  *M = int64_t(h->m.keys.size());
  if (keys) {
    if (cap < *M) return fail(ORACLE_EOVERFLOW, "capacity");
    std::copy(h->m.keys.begin(), h->m.keys.end(), keys);
  }
  return 0;
}

int oracle_get_state(oracle_mesh* h, double* u, int64_t cap) {
  if (!h) return fail(ORACLE_EINVAL, "null mesh");
  if (cap < int64_t(h->m.u.size())) return fail(ORACLE_EOVERFLOW, "capacity");
  std::copy(h->m.u.begin(), h->m.u.end(), u);
  return 0;
}

int oracle_set_state(oracle_mesh* h, const uint64_t* keys, int64_t M, const double* u) {
  if (!h) return fail(ORACLE_EINVAL, "null mesh");
  MeshO& m = h->m;
  std::vector<uint64_t> k(keys, keys + M);
  if (!complete(m.g, k)) return fail(ORACLE_EINVAL, "keys are not a complete linear tree");
  Conn cn;
  int rc = build_conn(m.g, k, cn);
  if (rc) return rc;
  m.keys.swap(k);
  m.conn = cn;
  m.u.assign(u, u + M * m.nv * m.N);
  return 0;
}

int oracle_get_conn(oracle_mesh* h, int32_t* nbr, int8_t* ftype, int8_t* slot, int64_t cap) {
  if (!h) return fail(ORACLE_EINVAL, "null mesh");
  int64_t S = int64_t(h->m.conn.nbr.size());
  if (cap < S) return fail(ORACLE_EOVERFLOW, "capacity");
  std::copy(h->m.conn.nbr.begin(), h->m.conn.nbr.end(), nbr);
  std::copy(h->m.conn.ftype.begin(), h->m.conn.ftype.end(), ftype);
  std::copy(h->m.conn.slot.begin(), h->m.conn.slot.end(), slot);
  return 0;
}

int oracle_set_time(oracle_mesh* h, double t) {
  if (!h) return fail(ORACLE_EINVAL, "null mesh");
  h->m.t = t;
  return 0;
}

int oracle_get_info(oracle_mesh* h, double* t, double* dt, int64_t* M, int64_t* step) {
  if (!h) return fail(ORACLE_EINVAL, "null mesh");
  if (t) *t = h->m.t;
  if (dt) *dt = h->m.dt;
  if (M) *M = int64_t(h->m.keys.size());
  if (step) *step = h->m.step;
  return 0;
}

}  // extern "C"
