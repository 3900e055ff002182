// fr_tree.cu -- linear-tree kernels (Sec. 3 and Sec. 4.1-4.2 of arXiv 2306.06744) on sm_103a:
// Morton encoding, linearisation, the adaptation edit, 2:1 balance by depth passes, old->new
// mapping and face connectivity.  Every generating step is count -> exclusive scan -> write at
// the scanned position, so outputs are deterministic and already in Morton order (no atomic
// counters, no retry on shared-memory overflow).
#include "fr_internal.cuh"

namespace frg {

namespace {

constexpr int TB = 256;
inline unsigned nblk(int64_t n, int b = TB) { return unsigned((n + b - 1) / b); }

template <int DIM>
__global__ void k_encode(const int32_t* __restrict__ boxes, int64_t n, uint64_t* __restrict__ keys,
                         KG g, int32_t* bad) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int d = boxes[4 * i];
  uint32_t x[3];
  bool ok = d >= 0 && d <= g.Dmax;
  for (int a = 0; a < DIM; ++a) {
    int32_t v = boxes[4 * i + 1 + a];
    ok = ok && v >= 0 && int64_t(v) < (int64_t(1) << g.Dmax);
    x[a] = uint32_t(v);
    if (ok) ok = (x[a] & (g.width(d) - 1u)) == 0u;
  }
  if (!ok) {
    atomicExch(bad, 1);
    keys[i] = 0;
    return;
  }
  keys[i] = g.make(interleave<DIM>(x), d);
}

template <int DIM>
__global__ void k_uniform(uint64_t* __restrict__ keys, int64_t count, KG g, int D) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < count) keys[i] = g.make(uint64_t(i) << (DIM * (g.Dmax - D)), D);
}

// keep[i] = no duplicate of and no descendant in the next key (sorted input: the subtree of an
// octant follows it contiguously, so checking the successor suffices)
template <int DIM>
__global__ void k_lin_count(const uint64_t* __restrict__ k, int64_t n, KG g, int32_t* __restrict__ cnt) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  bool drop = false;
  if (i + 1 < n) {
    uint64_t a = k[i], b = k[i + 1];
    drop = (a == b) || is_ancestor<DIM>(g, a, b);
  }
  cnt[i] = drop ? 0 : 1;
}

__global__ void k_compact(const uint64_t* __restrict__ k, const int32_t* __restrict__ cnt,
                          const int64_t* __restrict__ offs, int64_t n, uint64_t* __restrict__ out) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n && cnt[i]) out[offs[i]] = k[i];
}

// Adaptation edit (Sec. 4.1): action 0 keep, 1 refine, 2 head of a coarsened sibling group
// (becomes the parent), 3 other member of that group (removed).  Coarsening needs all 2^dim
// siblings present as consecutive leaves (raw IDs consecutive, Sec. 4.1) and all flagged -1.
template <int DIM>
__device__ __forceinline__ int edit_action(const uint64_t* __restrict__ k, const int8_t* __restrict__ flags,
                                           int64_t n, const KG& g, int Dbase, int64_t i) {
  constexpr int NC = 1 << DIM;
  const uint64_t key = k[i];
  const int d = g.depth(key);
  const int f = flags[i];
  if (f > 0 && d < g.Dmax) return 1;
  if (f < 0 && d > Dbase) {
    const int c = child_index<DIM>(g, key);
    const int64_t h = i - c;
    bool ok = h >= 0 && h + NC <= n;
    if (ok) {
      const uint64_t par = parent_key<DIM>(g, key);
      for (int s = 0; s < NC && ok; ++s)
        ok = k[h + s] == child_key<DIM>(g, par, s) && flags[h + s] < 0;
    }
    if (ok) return (c == 0) ? 2 : 3;
  }
  return 0;
}
__device__ __forceinline__ int edit_count(int a, int dim) { return a == 1 ? (1 << dim) : (a == 3 ? 0 : 1); }

template <int DIM>
__global__ void k_edit_count(const uint64_t* __restrict__ k, const int8_t* __restrict__ flags,
                             int64_t n, KG g, int Dbase, int8_t* __restrict__ act,
                             int32_t* __restrict__ cnt, int64_t* __restrict__ ctl,
                             int32_t* __restrict__ flags_out) {
  pdl_wait_then_release();
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i == 0) {  // the adaptation's control block and error flags start at zero
    for (int c = 0; c < CTL_SLOTS; ++c) ctl[c] = 0;
    if (flags_out) flags_out[0] = flags_out[1] = 0;
  }
  if (i >= n) return;
  const int a = edit_action<DIM>(k, flags, n, g, Dbase, i);
  act[i] = int8_t(a);
  cnt[i] = edit_count(a, DIM);
}

// The edit's actions and output counts with the tile-local exclusive scan of the counts in one
// launch: a block of 256 threads takes one tile of SCAN_TILE_ITEMS leaves (8 consecutive leaves
// per thread), writes each leaf's offset inside the tile and the tile's total to sums[block];
// k_edit_write adds the tile's base (offs_base).  Zeroes the control block like k_edit_count.
constexpr int EDIT_SCAN_T = 256, EDIT_SCAN_I = int(SCAN_TILE_ITEMS) / EDIT_SCAN_T;
template <int DIM>
__global__ void __launch_bounds__(EDIT_SCAN_T) k_edit_scan(const uint64_t* __restrict__ k,
                                                          const int8_t* __restrict__ flags, int64_t n, KG g,
                                                          int Dbase, int8_t* __restrict__ act,
                                                          int64_t* __restrict__ offs, int64_t* __restrict__ sums,
                                                          int64_t* __restrict__ ctl, int32_t* __restrict__ flags_out) {
  pdl_wait_then_release();
  __shared__ int32_t s_warp[EDIT_SCAN_T / 32];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  if (blockIdx.x == 0 && t == 0) {  // the adaptation's control block and error flags start at zero
    for (int c = 0; c < CTL_SLOTS; ++c) ctl[c] = 0;
    if (flags_out) flags_out[0] = flags_out[1] = 0;
  }
  const int64_t i0 = int64_t(blockIdx.x) * SCAN_TILE_ITEMS + int64_t(t) * EDIT_SCAN_I;
  int c[EDIT_SCAN_I], run = 0;
#pragma unroll
  for (int q = 0; q < EDIT_SCAN_I; ++q) {
    const int64_t i = i0 + q;
    c[q] = 0;
    if (i < n) {
      const int a = edit_action<DIM>(k, flags, n, g, Dbase, i);
      act[i] = int8_t(a);
      c[q] = edit_count(a, DIM);
    }
    run += c[q];
  }
  int incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int w = lane < EDIT_SCAN_T / 32 ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < EDIT_SCAN_T / 32) s_warp[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  int64_t o = int64_t(incl - run + (wid ? s_warp[wid - 1] : 0));
#pragma unroll
  for (int q = 0; q < EDIT_SCAN_I; ++q) {
    const int64_t i = i0 + q;
    if (i < n) offs[i] = o;
    o += c[q];
  }
  if (t == EDIT_SCAN_T - 1) sums[blockIdx.x] = s_warp[EDIT_SCAN_T / 32 - 1];
}

template <int DIM>
__global__ void k_edit_write(const uint64_t* __restrict__ k, const int8_t* __restrict__ act,
                             const Offs O, int64_t n, KG g, uint64_t* __restrict__ out,
                             unsigned long long* stats, int32_t* __restrict__ org, int8_t* __restrict__ otg,
                             const KeyIndex XO) {
  pdl_wait_then_release();
  int64_t grand;
  const int64_t base = offs_base(O, int64_t(blockIdx.x) * blockDim.x, &grand);
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t key = k[i];
  int64_t o = O.offs[i] + base;
  const int a = act[i];
  switch (a) {
    case 0:
      out[o] = key;
      XO.note(o, key);
      break;
    case 1:
      for (int c = 0; c < (1 << DIM); ++c) {
        const uint64_t ck = child_key<DIM>(g, key, c);
        out[o + c] = ck;
        XO.note(o + c, ck);
      }
      atomicAdd(&stats[0], 1ull);
      break;
    case 2: {
      const uint64_t pk = parent_key<DIM>(g, key);
      out[o] = pk;
      XO.note(o, pk);
      atomicAdd(&stats[1], 1ull);
      break;
    }
    default: break;
  }
  if (org && a != 3) {
    // the origin: this leaf (kept, refined) or the family's first child (fused)
    const int nc = a == 1 ? (1 << DIM) : 1;
    for (int c = 0; c < nc; ++c) {
      org[o + c] = int32_t(i);
      otg[o + c] = int8_t(a);
    }
  }
}

// 2:1 balance pass at depth D (Sec. 3.2, balance algorithm): every depth-D leaf looks up the
// leaf containing the anchor of each of its 3^dim-1 same-size neighbour boxes (periodic).  A
// containing leaf A coarser than D-1 is split along the path towards that box down to depth D-1;
// all 2^dim children of every level on the path are emitted.
template <int DIM>
struct Nofs {
  static constexpr int value = DIM == 2 ? 8 : 26;
};

template <int DIM>
__device__ __forceinline__ bool bal_query(const uint64_t* __restrict__ k, int64_t n, const KG& g,
                                          int D, int64_t i, int o, uint32_t* N, int* dA, int64_t* jA = nullptr,
                                          const uint64_t* s_tab = nullptr, int m = 0, int sh = 0) {
  uint64_t key = k[i];
  if (g.depth(key) != D) return false;
  int oo = o < (DIM == 2 ? 4 : 13) ? o : o + 1;  // skip the centre of the 3^dim stencil
  uint32_t x[3];
  deinterleave<DIM>(g.raw(key), x);
  uint32_t w = g.width(D), mask = (g.Dmax >= 32) ? 0xFFFFFFFFu : ((1u << g.Dmax) - 1u);
  for (int a = 0; a < DIM; ++a) {
    int off = (oo / (a == 0 ? 1 : (a == 1 ? 3 : 9))) % 3 - 1;
    N[a] = (x[a] + uint32_t(off) * w) & mask;  // periodic wrap on the 2^Dmax grid
  }
  int64_t j = bound_indexed<true>(k, n, cell_key<DIM>(g, N), s_tab, m, sh) - 1;
  if (j < 0) j = 0;  // only on an incomplete tree, which callers reject beforehand
  *dA = g.depth(k[j]);
  if (jA) *jA = j;
  return *dA < D - 1;
}

// The balance kernels read the leaf and octant counts from the adaptation's control block
// (CTL_* slots), so a whole adaptation can be issued without a host synchronisation; a pass whose
// octants exceed the capacity it was given is recorded in CTL_OVER, and it and all later passes
// leave the tree as it is, for the caller to finish with exact sizes.

// generated octants of the current pass that the merge uses: none after an overflow
__device__ __forceinline__ int64_t bal_nS(const int64_t* ctl, int64_t cap) {
  const int64_t G = ctl[CTL_G];
  return (ctl[CTL_OVER] != 0 || G > cap) ? 0 : G;
}

// A group of lanes per leaf (8 in 2D, a warp in 3D), one lane per neighbour box of the leaf's
// 3^dim-1 stencil: the lanes search in parallel and combine by warp shuffles, so the scan that
// places the generated octants runs over leaves, not over (leaf, neighbour) pairs.  Lanes past
// the leaf count (an upper bound of it sizes the grid) contribute zeros.
template <int DIM>
struct BalLanes {
  static constexpr int value = DIM == 2 ? 8 : 32;
};

// number of octants lane (i, o) generates, with the containing leaf's depth and the box
template <int DIM>
__device__ __forceinline__ int bal_lane(const uint64_t* __restrict__ k, int64_t n, const KG& g, int D,
                                        int64_t i, int o, uint32_t* N, int* dA, int64_t* jA = nullptr,
                                        const uint64_t* s_tab = nullptr, int m = 0, int sh = 0) {
  constexpr int NO = Nofs<DIM>::value;
  if (i >= n || o >= NO) return 0;
  return bal_query<DIM>(k, n, g, D, i, o, N, dA, jA, s_tab, m, sh) ? (D - 1 - *dA) << DIM : 0;
}

template <int DIM>
__global__ void k_bal_count(const uint64_t* __restrict__ k, const int64_t* __restrict__ ctl,
                            int64_t n_ub, KG g, int D, int32_t* __restrict__ cnt) {
  pdl_wait_then_release();
  constexpr int LPL = BalLanes<DIM>::value;
  const int64_t gt = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t i = gt / LPL;
  const int o = int(gt % LPL);
  const int64_t n = ctl[CTL_OVER] == 0 ? ctl[CTL_N] : 0;
  uint32_t N[3];
  int dA = 0;
  int c = i < n_ub ? bal_lane<DIM>(k, n, g, D, i, o, N, &dA) : 0;
#pragma unroll
  for (int w = LPL / 2; w > 0; w >>= 1) c += __shfl_xor_sync(0xffffffffu, c, w);
  if (o == 0 && i < n_ub) cnt[i] = c;
}

template <int DIM>
__global__ void k_bal_gen(const uint64_t* __restrict__ k, int64_t* __restrict__ ctl,
                          int64_t n_ub, KG g, int D, const Offs O,
                          uint64_t* __restrict__ out, int64_t cap) {
  pdl_wait_then_release();
  constexpr int LPL = BalLanes<DIM>::value;
  const int64_t gt = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t i = gt / LPL;
  const int o = int(gt % LPL);
  // the pass's octant count: from the tile totals (block 0 then stores it in ctl[CTL_G]) or,
  // after a full scan, from ctl[CTL_G]
  int64_t grand;
  const int64_t base = offs_base(O, int64_t(blockIdx.x) * (blockDim.x / LPL), &grand);
  const int64_t G = O.sums ? grand : ctl[CTL_G];
  const int64_t n = (ctl[CTL_OVER] == 0 && G > 0 && G <= cap) ? ctl[CTL_N] : 0;
  uint32_t N[3];
  int dA = 0;
  const int c = i < n_ub ? bal_lane<DIM>(k, n, g, D, i, o, N, &dA) : 0;
  // exclusive prefix of the counts among this leaf's lanes
  int incl = c;
#pragma unroll
  for (int w = 1; w < LPL; w <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, w, LPL);
    if (o >= w) incl += y;
  }
  if (c == 0) return;
  int64_t q = O.offs[i] + base + (incl - c);
  const uint64_t rawN = interleave<DIM>(N);
  for (int l = dA + 1; l <= D - 1; ++l) {
    const uint64_t span = vol_raw<DIM>(g, l - 1);
    const uint64_t anc = g.make(rawN / span * span, l - 1);  // ancestor of the box at depth l-1
    for (int ch = 0; ch < (1 << DIM); ++ch) out[q++] = child_key<DIM>(g, anc, ch);
  }
}

// Sort of the generated octants (at most SMALL_SORT_MAX) inside one block: bitonic network over a
// power-of-two padded array in shared memory (padding = all-ones keys, which sort last and are
// not written back).  Exchanges closer than 32 elements stay inside one warp and need only a
// warp barrier.  Up to RANK_SORT_MAX keys a rank sort is used instead (one pass over the keys).
// Also the capacity check of the pass: an oversized pass is recorded, not sorted.
constexpr int SMALL_SORT_MAX = 4096, RANK_SORT_MAX = 256;
__global__ void __launch_bounds__(1024) k_sort_small(uint64_t* __restrict__ keys, int64_t* __restrict__ ctl,
                                                     int64_t cap, int D) {
  pdl_wait_then_release();
  __shared__ uint64_t sk[SMALL_SORT_MAX];
  if (ctl[CTL_OVER] != 0) return;
  const int64_t n = ctl[CTL_G];
  if (n > cap || n > SMALL_SORT_MAX) {
    if (threadIdx.x == 0) ctl[CTL_OVER] = D;
    return;
  }
  if (n == 0) return;
  if (n <= RANK_SORT_MAX) {
    // rank sort: each key's position is the number of smaller keys plus the equal keys before it
    // (n^2 comparisons on one SM: cheaper than the network's log^2 barriers only for small n)
    const int t = threadIdx.x;
    uint64_t mine = 0;
    if (t < n) mine = sk[t] = keys[t];
    __syncthreads();
    if (t < n) {
      int r = 0;
      for (int j = 0; j < n; ++j) {
        const uint64_t o = sk[j];
        r += (o < mine) || (o == mine && j < t);
      }
      keys[r] = mine;
    }
    return;
  }
  int P = 1;
  while (P < n) P <<= 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x) sk[i] = i < n ? keys[i] : ~0ull;
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        int l = i ^ j;
        if (l > i) {
          uint64_t a = sk[i], b = sk[l];
          bool up = (i & k) == 0;
          if ((a > b) == up) {
            sk[i] = b;
            sk[l] = a;
          }
        }
      }
      const int next_j = j > 1 ? j >> 1 : k;  // partner distance of the next stage
      if (j >= 32 || next_j >= 32)
        __syncthreads();
      else
        __syncwarp();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) keys[i] = sk[i];
}

// Merge of the sorted generated octants S (duplicates and ancestors still present) into the tree.
// Every generated octant lies strictly inside one current leaf, and the octants inside a leaf
// cover it once linearised (path splitting emits all 2^dim children at each level), so a leaf
// with a non-empty range [lo, hi) is replaced by the linearised octants of that range and any
// other leaf is kept.  Linearisation keeps S[r] unless S[r+1] equals it or lies inside it; a set
// already linearised (`linearised`) is copied range by range.
template <int DIM>
__device__ __forceinline__ bool lin_keep(const uint64_t* __restrict__ S, int64_t nS, const KG& g, int64_t r) {
  if (r + 1 >= nS) return true;
  uint64_t a = S[r], b = S[r + 1];
  return !(a == b || is_ancestor<DIM>(g, a, b));
}
template <int DIM>
__global__ void k_merge_count(const uint64_t* __restrict__ k, int64_t* __restrict__ ctl,
                              int64_t n_ub, const uint64_t* __restrict__ S, int64_t cap, KG g,
                              bool linearised, int32_t* __restrict__ cnt, int64_t* __restrict__ lo_out) {
  pdl_wait_then_release();
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_ub) return;
  const int64_t nS = bal_nS(ctl, cap);
  if (i == 0 && nS > 0) ctl[CTL_PASSES] += 1;  // a pass that changes the tree
  if (i >= ctl[CTL_N]) {
    cnt[i] = 0;
    lo_out[i] = -1;
    return;
  }
  uint64_t key = k[i];
  int64_t lo = lower_bound_dev(S, nS, key);
  int64_t hi = lower_bound_dev(S, nS, key_end<DIM>(g, key));
  int32_t c = 1;
  if (hi > lo) {
    if (linearised) {
      c = int32_t(hi - lo);
    } else {
      c = 0;
      for (int64_t r = lo; r < hi; ++r) c += lin_keep<DIM>(S, nS, g, r);
    }
  }
  cnt[i] = c;
  lo_out[i] = hi > lo ? lo : -1;  // -1: the leaf is kept as it is
}
// runs after the merged count has replaced ctl[CTL_N]: rows past the old count have cnt 0
template <int DIM>
__global__ void k_merge_write(const uint64_t* __restrict__ k, const int64_t* __restrict__ ctl,
                              int64_t n_ub, const uint64_t* __restrict__ S, int64_t cap, KG g,
                              bool linearised, const int32_t* __restrict__ cnt,
                              const int64_t* __restrict__ lo, const Offs O,
                              uint64_t* __restrict__ out) {
  pdl_wait_then_release();
  int64_t grand;
  const int64_t base = offs_base(O, int64_t(blockIdx.x) * blockDim.x, &grand);
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_ub) return;
  const int c = cnt[i];
  if (c == 0) return;
  int64_t o = O.offs[i] + base, l = lo[i];
  if (l < 0) {
    out[o] = k[i];
    return;
  }
  const int64_t nS = bal_nS(ctl, cap), end = o + c;
  if (linearised) {
    for (int64_t r = l; o < end; ++r) out[o++] = S[r];
  } else {
    for (int64_t r = l; o < end; ++r)
      if (lin_keep<DIM>(S, nS, g, r)) out[o++] = S[r];
  }
}

// ---- balance pass issued without host synchronisation: generate -> sort -> merge ----
// The octants of a pass are placed by a warp-aggregated atomic counter: their order does not
// matter, because they are sorted next and equal keys are indistinguishable, so the tree stays
// bit-exact.  The sort kernel, which holds the whole sorted set, also computes where every leaf
// lands in the merged tree: a leaf that holds octants becomes its k >= 1 linearised octants, so
// the leaves before it shift by the sum of (k - 1) over the leaves holding octants before it,
// P[r] = sum over the sorted octants s < r of (kept(s) - first octant of its leaf(s)).  The merge
// then needs no count and no scan over the leaves.
// With `packed` (when the key's bits and PACK_BITS fit 64), each octant is stored as
// key << PACK_BITS | index of the leaf that contains it: sorting the packed values sorts the keys
// (equal keys lie in the same leaf), and the sort kernel then reads the containing leaf instead of
// searching for it.
constexpr int PACK_BITS = 21;  // leaf indices below 2^21 (meshes of this path hold at most 2^20)
template <int DIM>
__global__ void k_bal_gen_fast(const uint64_t* __restrict__ k, int64_t* __restrict__ ctl, int64_t n_ub, KG g,
                               int D, uint64_t* __restrict__ out, int64_t cap, bool packed, int sn, int sg,
                               const KeyIndex X) {
  pdl_wait_then_release();
  __shared__ uint64_t s_tab[KEY_INDEX_MAX];
  constexpr int LPL = BalLanes<DIM>::value;
  constexpr int NC = 1 << DIM;
  const int64_t gt = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t i = gt / LPL;
  const int o = int(gt % LPL);
  const int64_t n = ctl[CTL_OVER] == 0 ? ctl[sn] : 0;
  // the key index is staged only by blocks that hold a depth-D leaf (the others search nothing)
  const bool deep = i < n_ub && i < n && g.depth(k[i]) == D;
  int m = 0;
  if (__syncthreads_or(deep)) m = stage_key_index(X, n, s_tab);
  uint32_t N[3];
  int dA = 0;
  int64_t jA = 0;
  const bool gen = deep && bal_lane<DIM>(k, n, g, D, i, o, N, &dA, &jA, s_tab, m, X.sh) > 0;
  // A lane emits the 2^dim children of its box's ancestor at each depth l-1, l = dA+1 .. D-1.
  // Lanes of a warp whose boxes share that ancestor (neighbouring leaves looking into the same
  // coarse leaf) would emit the same octants: per depth only the lowest such lane emits them, so
  // the set of octants is unchanged and the sort and merge see fewer copies.
  const int lane = int(threadIdx.x & 31);
  const int l0 = int(__reduce_min_sync(0xffffffffu, unsigned(gen ? dA + 1 : D)));
  const uint64_t rawN = gen ? interleave<DIM>(N) : 0ull;
  uint32_t lead = 0;  // bit l - l0: this lane emits depth l's octants
  int c = 0;
  for (int l = l0; l <= D - 1; ++l) {
    const bool act = gen && l > dA;
    const uint64_t span = vol_raw<DIM>(g, l - 1);
    // an ancestor key never equals the all-ones value of the lanes that emit nothing
    const uint64_t anc = act ? g.make(rawN / span * span, l - 1) : ~0ull;
    const unsigned same = __match_any_sync(0xffffffffu, anc);
    if (act && lane == __ffs(same) - 1) {
      lead |= 1u << (l - l0);
      c += NC;
    }
  }
  // every lane of the warp takes part: inclusive prefix of the counts, one atomic per warp
  int incl = c;
#pragma unroll
  for (int w = 1; w < 32; w <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, w);
    if (lane >= w) incl += y;
  }
  const int tot = __shfl_sync(0xffffffffu, incl, 31);
  unsigned long long base = 0;
  if (lane == 31 && tot > 0) base = atomicAdd(reinterpret_cast<unsigned long long*>(ctl + sg), (unsigned long long)tot);
  base = __shfl_sync(0xffffffffu, base, 31);
  if (c == 0) return;
  int64_t q = int64_t(base) + (incl - c);
  for (int l = l0; l <= D - 1; ++l) {
    if (!((lead >> (l - l0)) & 1u)) continue;
    const uint64_t span = vol_raw<DIM>(g, l - 1);
    const uint64_t anc = g.make(rawN / span * span, l - 1);
    for (int ch = 0; ch < NC; ++ch, ++q)
      if (q < cap) {  // past the capacity: counted, not stored
        const uint64_t ck = child_key<DIM>(g, anc, ch);
        out[q] = packed ? (ck << PACK_BITS) | uint64_t(jA) : ck;
      }
  }
}

// Sort of a pass's nS generated values (at most SMALL_SORT_MAX, nS > 0) by one block of 1024
// threads into sk: a rank sort up to RANK_SORT_MAX values, else a bitonic network over the
// power-of-two padded array (padding all-ones, sorted last); exchanges closer than 32 elements
// stay inside one warp and need only a warp barrier.  Ends with a block barrier.
__device__ __forceinline__ void block_sort_1024(uint64_t* sk, const uint64_t* __restrict__ S, int nS) {
  const int t = threadIdx.x;
  if (nS <= RANK_SORT_MAX) {
    // rank sort: each key's position is the number of smaller keys plus the equal keys before it
    uint64_t mine = 0;
    int r = 0;
    if (t < nS) mine = sk[t] = S[t];
    __syncthreads();
    if (t < nS)
      for (int j = 0; j < nS; ++j) {
        const uint64_t o = sk[j];
        r += (o < mine) || (o == mine && j < t);
      }
    __syncthreads();  // every rank is taken before the keys move
    if (t < nS) sk[r] = mine;
  } else {
    int Pw = 1;
    while (Pw < nS) Pw <<= 1;
    // up to four loads in flight per thread (Pw <= 4 x blockDim)
    uint64_t v[SMALL_SORT_MAX / 1024];
#pragma unroll
    for (int q = 0; q < SMALL_SORT_MAX / 1024; ++q) {
      const int i = t + q * 1024;
      v[q] = i < nS ? S[i] : ~0ull;
    }
#pragma unroll
    for (int q = 0; q < SMALL_SORT_MAX / 1024; ++q)
      if (t + q * 1024 < Pw) sk[t + q * 1024] = v[q];
    __syncthreads();
    for (int kk = 2; kk <= Pw; kk <<= 1) {
      for (int j = kk >> 1; j > 0; j >>= 1) {
        for (int i = t; i < Pw; i += blockDim.x) {
          const int l = i ^ j;
          if (l > i) {
            const uint64_t a = sk[i], b = sk[l];
            const bool up = (i & kk) == 0;
            if ((a > b) == up) {
              sk[i] = b;
              sk[l] = a;
            }
          }
        }
        const int next_j = j > 1 ? j >> 1 : kk;
        if (j >= 32 || next_j >= 32)
          __syncthreads();
        else
          __syncwarp();
      }
    }
  }
  __syncthreads();
}

// one block: sorts the pass's octants, computes the merge shifts P[0..nS] and the merged leaf
// count, and prepares the control block for the merge (CTL_NPREV, CTL_GS) and the next pass
// (CTL_G zeroed).  An oversized pass, or any pass after one, merges nothing.
template <int DIM>
__global__ void __launch_bounds__(1024) k_sort_annot(uint64_t* __restrict__ S, int64_t* __restrict__ ctl,
                                                     int64_t cap, int D, const uint64_t* __restrict__ k, KG g,
                                                     int32_t* __restrict__ P, bool packed) {
  pdl_wait_then_release();
  __shared__ uint64_t sk[SMALL_SORT_MAX];
  __shared__ int32_t wsum[32];
  const int t = threadIdx.x;
  const int64_t n = ctl[CTL_N];
  const int64_t G = ctl[CTL_G];
  const bool over = ctl[CTL_OVER] != 0 || G > cap || G > SMALL_SORT_MAX;
  __syncthreads();  // every thread has read the control block before thread 0 rewrites it
  if (over || G == 0) {
    if (t == 0) {
      if (ctl[CTL_OVER] == 0 && G > 0) ctl[CTL_OVER] = D;
      ctl[CTL_NPREV] = n;
      ctl[CTL_GS] = 0;
      ctl[CTL_G] = 0;
    }
    return;
  }
  const int nS = int(G);
  block_sort_1024(sk, S, nS);  // the sorted octants are in sk
  // per thread 4 consecutive octants r = 4t .. 4t+3: kept(r) - first(r), with first(r) when the
  // containing leaf of r differs from that of r - 1
  // (packed: the containing leaf is the value's low bits, the key its high bits; the sorted keys
  // are written back to S unpacked)
  const uint64_t lmask = (1ull << PACK_BITS) - 1;
  auto leaf_of = [&](int r) -> int64_t {
    return packed ? int64_t(sk[r] & lmask) : upper_bound_dev(k, n, sk[r]) - 1;
  };
  auto keep_of = [&](int r) -> bool {
    if (!packed) return lin_keep<DIM>(sk, nS, g, r);
    if (r + 1 >= nS) return true;
    const uint64_t a = sk[r] >> PACK_BITS, b = sk[r + 1] >> PACK_BITS;
    return !(a == b || is_ancestor<DIM>(g, a, b));
  };
  int v[4], sum = 0;
  int64_t prev_leaf = -1;
  if (4 * t < nS && 4 * t > 0) prev_leaf = leaf_of(4 * t - 1);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = 4 * t + q;
    v[q] = 0;
    if (r < nS) {
      const int64_t leaf = leaf_of(r);
      v[q] = int(keep_of(r)) - int(leaf != prev_leaf);
      prev_leaf = leaf;
    }
    sum += v[q];
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = 4 * t + q;
    if (r < nS) S[r] = packed ? sk[r] >> PACK_BITS : sk[r];
  }
  // block-wide exclusive scan of the per-thread sums
  const int lane = t & 31, wid = t >> 5;
  int incl = sum;
#pragma unroll
  for (int w = 1; w < 32; w <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, w);
    if (lane >= w) incl += y;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const int x = lane < int(blockDim.x >> 5) ? wsum[lane] : 0;
    int wi = x;
#pragma unroll
    for (int w = 1; w < 32; w <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, wi, w);
      if (lane >= w) wi += y;
    }
    wsum[lane] = wi - x;  // exclusive prefix of the warp totals
  }
  __syncthreads();
  int run = wsum[wid] + incl - sum;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = 4 * t + q;
    if (r < nS) P[r] = run;
    run += v[q];
    if (r == nS - 1) {
      P[nS] = run;  // total shift: the merged tree holds n + P[nS] leaves
      ctl[CTL_NPREV] = n;
      ctl[CTL_N] = n + run;
      ctl[CTL_GS] = nS;
      ctl[CTL_G] = 0;
      ctl[CTL_PASSES] += 1;
    }
  }
}

// the sorted octants (at most SMALL_SORT_MAX) are staged in shared memory: every leaf searches them
__device__ __forceinline__ int lower_bound_sh(const uint64_t* a, int n, uint64_t v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}
// With oi/ti (origin and relation of each leaf to the tree before the edit, tree_edit): the same
// for the merged tree into oo/to.  An octant inside leaf X lies inside X's origin (relation 1),
// unless X is a fused parent: then the octant is, or lies inside, the old child that contains it.
template <int DIM>
__global__ void k_merge_fast(const uint64_t* __restrict__ k, const int64_t* __restrict__ ctl, int64_t n_ub,
                             const uint64_t* __restrict__ S, const int32_t* __restrict__ P, KG g,
                             uint64_t* __restrict__ out, const int32_t* __restrict__ oi,
                             const int8_t* __restrict__ ti, int32_t* __restrict__ oo, int8_t* __restrict__ to) {
  pdl_wait_then_release();
  __shared__ uint64_t sS[SMALL_SORT_MAX];
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t n = ctl[CTL_NPREV];
  const int nS = int(ctl[CTL_GS]);  // at most SMALL_SORT_MAX (the sort kernel's capacity check)
  if (int64_t(blockIdx.x) * blockDim.x >= n) return;  // the whole block is past the leaves
  // eight loads in flight per thread before their stores
  for (int r0 = threadIdx.x; r0 < nS; r0 += 8 * blockDim.x) {
    uint64_t v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int r = r0 + q * int(blockDim.x);
      v[q] = r < nS ? S[r] : 0ull;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int r = r0 + q * int(blockDim.x);
      if (r < nS) sS[r] = v[q];
    }
  }
  __syncthreads();
  if (i >= n_ub || i >= n) return;
  const uint64_t key = k[i];
  const int32_t src = oo ? oi[i] : 0;
  const int tag = oo ? ti[i] : 0;
  if (nS == 0) {
    out[i] = key;
    if (oo) {
      oo[i] = src;
      to[i] = int8_t(tag);
    }
    return;
  }
  const int64_t lo = lower_bound_sh(sS, nS, key);
  const int64_t hi = lower_bound_sh(sS, nS, key_end<DIM>(g, key));
  int64_t o = i + P[lo];
  if (hi == lo) {
    out[o] = key;
    if (oo) {
      oo[o] = src;
      to[o] = int8_t(tag);
    }
    return;
  }
  const int d1 = g.depth(key) + 1;
  for (int64_t r = lo; r < hi; ++r)
    if (lin_keep<DIM>(sS, nS, g, r)) {
      const uint64_t y = sS[r];
      out[o] = y;
      if (oo) {
        if (tag == 2) {
          const uint64_t span = vol_raw<DIM>(g, d1);
          const int c = child_index<DIM>(g, g.make(g.raw(y) / span * span, d1));
          oo[o] = src + c;
          to[o] = int8_t(g.depth(y) == d1 ? 0 : 1);
        } else {
          oo[o] = src;
          to[o] = 1;
        }
      }
      ++o;
    }
}

// lower bound of key v among packed values (key << PACK_BITS | containing leaf), by their keys
__device__ __forceinline__ int lower_bound_packed(const uint64_t* a, int n, uint64_t v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((a[mid] >> PACK_BITS) < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}
// A balance pass issued without synchronisation whose octants carry their containing leaf
// (packed), in two launches instead of three: every block of the merge sorts the pass's octants
// itself in shared memory and computes the shifts P as k_sort_annot does (the per-leaf merge then
// follows k_merge_fast), over a grid-stride range of leaves.  The leaf count before the pass is
// read from slot si and the octant count from slot sg; block 0 writes the merged count to slot so,
// zeroes slot sg_next (the next pass's octant counter) and records an oversized pass in CTL_OVER
// (such a pass, and every later one, copies the tree).  No block reads a slot that block 0 writes
// in the same launch, except CTL_OVER, whose new value leads every block to the same decision.
template <int DIM>
__global__ void __launch_bounds__(1024) k_merge_sorted(const uint64_t* __restrict__ k, int64_t* __restrict__ ctl,
                                                       int64_t n_ub, const uint64_t* __restrict__ S, int64_t cap,
                                                       int D, int si, int sg, int so, int sg_next, KG g,
                                                       uint64_t* __restrict__ out, const int32_t* __restrict__ oi,
                                                       const int8_t* __restrict__ ti, int32_t* __restrict__ oo,
                                                       int8_t* __restrict__ to, const KeyIndex XO) {
  pdl_wait_then_release();
  __shared__ uint64_t sk[SMALL_SORT_MAX];
  __shared__ int16_t sP[SMALL_SORT_MAX + 1];  // |P| <= SMALL_SORT_MAX
  __shared__ int32_t wsum[32];
  const int t = threadIdx.x;
  const int64_t n = ctl[si];
  const int64_t G = ctl[sg];
  const bool big = G > cap || G > SMALL_SORT_MAX;
  const int nS = (ctl[CTL_OVER] != 0 || big) ? 0 : int(G);
  const int64_t nn = n < n_ub ? n : n_ub;
  if (blockIdx.x != 0 && int64_t(blockIdx.x) * blockDim.x >= nn) return;  // no leaves here
  const uint64_t lmask = (1ull << PACK_BITS) - 1;
  // octant r is kept by the linearisation unless the next one equals it or lies inside it
  auto keep_of = [&](int r) -> bool {
    if (r + 1 >= nS) return true;
    const uint64_t a = sk[r] >> PACK_BITS, b = sk[r + 1] >> PACK_BITS;
    return !(a == b || is_ancestor<DIM>(g, a, b));
  };
  int total = 0;
  if (nS > 0) {
    block_sort_1024(sk, S, nS);
    // per thread 4 consecutive octants r = 4t .. 4t+3: kept(r) - first(r), first(r) when the
    // containing leaf of r differs from that of r - 1; exclusive block scan into sP
    int v[4], sum = 0;
    uint64_t prev_leaf = ~0ull;
    if (4 * t < nS && 4 * t > 0) prev_leaf = sk[4 * t - 1] & lmask;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = 4 * t + q;
      v[q] = 0;
      if (r < nS) {
        const uint64_t leaf = sk[r] & lmask;
        v[q] = int(keep_of(r)) - int(leaf != prev_leaf);
        prev_leaf = leaf;
      }
      sum += v[q];
    }
    const int lane = t & 31, wid = t >> 5;
    int incl = sum;
#pragma unroll
    for (int w = 1; w < 32; w <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, w);
      if (lane >= w) incl += y;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      const int x = lane < int(blockDim.x >> 5) ? wsum[lane] : 0;
      int wi = x;
#pragma unroll
      for (int w = 1; w < 32; w <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, wi, w);
        if (lane >= w) wi += y;
      }
      wsum[lane] = wi - x;  // exclusive prefix of the warp totals
    }
    __syncthreads();
    int run = wsum[wid] + incl - sum;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = 4 * t + q;
      if (r < nS) sP[r] = int16_t(run);
      run += v[q];
      if (r == nS - 1) sP[nS] = int16_t(run);  // total shift: n + sP[nS] leaves after the merge
    }
    __syncthreads();
    total = sP[nS];
  }
  if (blockIdx.x == 0 && t == 0) {
    if (big && ctl[CTL_OVER] == 0) ctl[CTL_OVER] = D;
    ctl[so] = n + total;
    ctl[sg_next] = 0;
    if (nS > 0) ctl[CTL_PASSES] += 1;
  }
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + t; i < nn; i += int64_t(gridDim.x) * blockDim.x) {
    const uint64_t key = k[i];
    const int32_t src = oo ? oi[i] : 0;
    const int tag = oo ? ti[i] : 0;
    int lo = 0, hi = 0;
    if (nS > 0) {
      lo = lower_bound_packed(sk, nS, key);
      hi = lower_bound_packed(sk, nS, key_end<DIM>(g, key));
    }
    int64_t o = i + (nS > 0 ? int64_t(sP[lo]) : 0);
    if (hi == lo) {
      out[o] = key;
      XO.note(o, key);
      if (oo) {
        oo[o] = src;
        to[o] = int8_t(tag);
      }
      continue;
    }
    const int d1 = g.depth(key) + 1;
    for (int r = lo; r < hi; ++r)
      if (keep_of(r)) {
        const uint64_t y = sk[r] >> PACK_BITS;
        out[o] = y;
        XO.note(o, y);
        if (oo) {
          if (tag == 2) {
            const uint64_t span = vol_raw<DIM>(g, d1);
            const int c = child_index<DIM>(g, g.make(g.raw(y) / span * span, d1));
            oo[o] = src + c;
            to[o] = int8_t(g.depth(y) == d1 ? 0 : 1);
          } else {
            oo[o] = src;
            to[o] = 1;
          }
        }
        ++o;
      }
  }
}

// Old->new mapping (Sec. 4.2, mapping algorithm) by one lower bound per new leaf.
template <int DIM>
__global__ void k_map(const uint64_t* __restrict__ old, int64_t no, const uint64_t* __restrict__ nw,
                      int64_t nn_ub, const int64_t* __restrict__ d_nn, KG g, int32_t* __restrict__ src,
                      int8_t* __restrict__ tag, int32_t* bad) {
  pdl_wait_then_release();
  int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= nn_ub || (d_nn && j >= *d_nn)) return;
  map_leaf<DIM>(old, no, nw[j], g, src + j, tag + j, bad);
}

// Face connectivity (Sec. 3.3): same-depth face-neighbour box, point location of its anchor.
template <int DIM>
__global__ void k_conn(const uint64_t* __restrict__ k, int64_t n_ub, const int64_t* __restrict__ d_n, KG g,
                       int32_t* __restrict__ nbr, int8_t* __restrict__ ftype, int8_t* __restrict__ slot,
                       int32_t* __restrict__ contrib, int32_t* bad, int64_t* __restrict__ fcnt,
                       const FaceLists L) {
  pdl_wait_then_release();
  constexpr int NFC = 2 * DIM;
  // with fcnt: the block holds whole leaves (blockDim a multiple of 2*dim) and also writes each
  // leaf's face-list counts, conforming faces it owns (its + faces) low, coarse sides of hanging
  // faces high; leaves past the count get zero
  __shared__ int s_cnt[2 * 256 / NFC + 2];
  __shared__ uint64_t s_tab[KEY_INDEX_MAX];
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t n = d_n ? *d_n : n_ub;
  // blocks past the leaf count (the grid is sized by a bound of it) search nothing
  const int m = int64_t(blockIdx.x) * blockDim.x < n * NFC ? stage_key_index(L.index, n, s_tab) : 0;
  const int sh = L.index.sh;
  const int lt = int(threadIdx.x) / NFC;
  if (fcnt && int(threadIdx.x) % NFC == 0) s_cnt[2 * lt] = s_cnt[2 * lt + 1] = 0;
  if (fcnt) __syncthreads();
  const bool act = t < n_ub * NFC && t < n * NFC;
  int type = -1;
  int32_t cv[4];  // the coarse side's contributors of a hanging face (fine leaves by slot)
  const int f = int(t % NFC);
  if (act) {
    const int64_t e = t / NFC;
    const int axis = f >> 1, side = f & 1;
    const uint64_t key = k[e];
    const int d = g.depth(key);
    uint32_t x[3], N[3];
    deinterleave<DIM>(g.raw(key), x);
    const uint32_t w = g.width(d), mask = (g.Dmax >= 32) ? 0xFFFFFFFFu : ((1u << g.Dmax) - 1u);
    for (int a = 0; a < DIM; ++a) N[a] = x[a];
    N[axis] = (x[axis] + (side ? w : (0u - w))) & mask;
    const uint64_t kN = g.make(interleave<DIM>(N), d);
    int64_t j = bound_indexed<true>(k, n, cell_key<DIM>(g, N), s_tab, m, sh) - 1;
    if (j < 0) j = 0;
    const uint64_t kj = k[j];
    const int dj = g.depth(kj);
    if (kj == kN) {
      nbr[t] = int32_t(j);
      ftype[t] = 0;
      slot[t] = -1;
      type = 0;
    } else if (dj < d) {
      if (dj != d - 1) atomicExch(bad, 1);
      nbr[t] = int32_t(j);
      ftype[t] = 1;
      int c = child_index<DIM>(g, key), sl = 0, sh = 0;
      for (int b = 0; b < DIM; ++b)
        if (b != axis) sl |= ((c >> b) & 1) << sh++;
      slot[t] = int8_t(sl);
      type = 1;
    } else {
      ftype[t] = 2;
      slot[t] = 0;
      type = 2;
      int first = -1;
      cv[2] = cv[3] = -1;  // 2 contributors in 2D
      for (int c = 0; c < (1 << DIM); ++c) {
        if (((c >> axis) & 1) != (side ? 0 : 1)) continue;
        uint64_t kc = child_key<DIM>(g, kN, c);
        int64_t q = bound_indexed<false>(k, n, kc, s_tab, m, sh);
        if (q >= n || k[q] != kc) {
          atomicExch(bad, 1);
          q = 0;
        }
        int sl = 0, sb = 0;
        for (int b = 0; b < DIM; ++b)
          if (b != axis) sl |= ((c >> b) & 1) << sb++;
        if (sl == 0) first = int(q);
        cv[sl] = int32_t(q);
      }
      if (contrib)
        for (int r = 0; r < 4; ++r) contrib[t * 4 + r] = cv[r];
      nbr[t] = first;
    }
  }
  if (L.conf) {
    // the face lists themselves: a block's conforming faces it owns (its + faces) and coarse
    // sides of hanging faces, in (leaf, face) order, appended at a base that one atomic per block
    // takes from the packed counter (conforming low, hanging high).  The order of the blocks'
    // ranges is arbitrary; every face's fluxes are computed and written by that face alone.
    __shared__ int s_wc[8], s_wh[8];
    __shared__ unsigned long long s_base;
    const bool ec = (f & 1) && type == 0, eh = type == 2;
    const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    const unsigned bc = __ballot_sync(0xFFFFFFFFu, ec), bh = __ballot_sync(0xFFFFFFFFu, eh);
    const unsigned below = (1u << lane) - 1u;
    if (lane == 0) {
      s_wc[wid] = __popc(bc);
      s_wh[wid] = __popc(bh);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long tc = 0, th = 0;
      for (unsigned w = 0; w < (blockDim.x + 31u) / 32u; ++w) {
        const int a = s_wc[w], b = s_wh[w];
        s_wc[w] = int(tc);
        s_wh[w] = int(th);
        tc += unsigned(a);
        th += unsigned(b);
      }
      s_base = (tc | th) ? atomicAdd(L.count, tc | (th << 32)) : 0ull;
    }
    __syncthreads();
    const unsigned long long base = s_base;
    const int64_t e = t / NFC;
    if (ec) L.conf[int64_t(base & 0xFFFFFFFFull) + s_wc[wid] + __popc(bc & below)] = int32_t((e << 2) | (f >> 1));
    if (eh) {
      const int64_t h = int64_t(base >> 32) + s_wh[wid] + __popc(bh & below);
      L.hang[h] = int32_t((e << 3) | f);
      for (int r = 0; r < 4; ++r) L.hcon[h * 4 + r] = cv[r];
    }
    if (L.pub) {
      // the last block to finish publishes the counts (every block's atomics precede its fence)
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(L.done, 1ull) == gridDim.x - 1ull) {
          __threadfence();
          for (int w = 0; w < L.nwords; ++w)
            L.pub[w] = *reinterpret_cast<const volatile int64_t*>(L.words + w);
          __threadfence_system();
          *reinterpret_cast<volatile int64_t*>(L.pub + L.nwords) = L.seq;
          __threadfence_system();
        }
      }
    }
  }
  if (!fcnt) return;
  if ((f & 1) && type == 0) atomicAdd(&s_cnt[2 * lt], 1);
  if (type == 2) atomicAdd(&s_cnt[2 * lt + 1], 1);
  __syncthreads();
  const int64_t e = t / NFC;
  if (f == 0 && e < n_ub) fcnt[e] = int64_t(s_cnt[2 * lt]) | (int64_t(s_cnt[2 * lt + 1]) << 32);
}

template <int DIM>
__global__ void k_validate(const uint64_t* __restrict__ k, int64_t n, KG g, int Dlo, int Dhi,
                           int32_t* bad) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t key = k[i];
  int d = g.depth(key);
  uint64_t total = 1ull << (DIM * g.Dmax);
  bool ok = d >= Dlo && d <= Dhi && d <= g.Dmax;
  if (ok) {
    uint64_t raw = g.raw(key), v = vol_raw<DIM>(g, d);
    ok = (raw % v) == 0 && raw < total;
    uint64_t next = (i + 1 < n) ? g.raw(k[i + 1]) : total;
    ok = ok && raw + v == next;
    if (i == 0) ok = ok && raw == 0;
  }
  if (!ok) atomicExch(bad, 1);
}

// Tree completion (Sec. 3.1): the finest cell of each point becomes a seed octant; between two
// consecutive seeds (and before the first / after the last) the Morton interval of finest cells
// is covered greedily by the largest aligned octants that fit, never coarser than Dmin.  This is
// the coarsest complete tree holding the seeds as leaves, and it comes out already sorted.
template <int DIM>
__global__ void k_pts_encode(const double* __restrict__ pts, int64_t n, double L, KG g,
                             uint64_t* __restrict__ keys) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double side = double(1ull << g.Dmax);
  uint32_t x[3] = {0, 0, 0};
  for (int a = 0; a < DIM; ++a) {
    double c = floor(pts[i * DIM + a] / L * side);
    x[a] = c < 0.0 ? 0u : (c >= side ? uint32_t(side) - 1u : uint32_t(c));
  }
  keys[i] = cell_key<DIM>(g, x);
}

// greedy decomposition of the raw-ID interval [lo, hi]; emits (raw, depth) when out != null
template <int DIM>
__device__ __forceinline__ int64_t gap_blocks(uint64_t lo, uint64_t hi_excl, const KG& g, int Dmin,
                                              uint64_t* out) {
  int64_t cnt = 0;
  const int kmax = g.Dmax - Dmin;
  while (lo < hi_excl) {
    int k = 0;
    while (k < kmax) {
      uint64_t span = 1ull << (DIM * (k + 1));
      if ((lo & (span - 1)) != 0 || lo + span > hi_excl) break;
      ++k;
    }
    if (out) out[cnt] = g.make(lo, g.Dmax - k);
    ++cnt;
    lo += 1ull << (DIM * k);
  }
  return cnt;
}

template <int DIM>
__device__ __forceinline__ void gap_bounds(const uint64_t* S, int64_t nS, int64_t t, const KG& g,
                                           uint64_t* lo, uint64_t* hi_excl) {
  *lo = t == 0 ? 0ull : g.raw(S[t - 1]) + vol_raw<DIM>(g, g.depth(S[t - 1]));
  *hi_excl = t == nS ? (1ull << (DIM * g.Dmax)) : g.raw(S[t]);
}

template <int DIM>
__global__ void k_gap_count(const uint64_t* __restrict__ S, const int64_t* __restrict__ d_nS,
                            int64_t ncap, KG g, int Dmin, int32_t* __restrict__ cnt) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t > ncap) return;
  const int64_t nS = *d_nS;
  if (t > nS) {
    cnt[t] = 0;
    return;
  }
  uint64_t lo, hi;
  gap_bounds<DIM>(S, nS, t, g, &lo, &hi);
  cnt[t] = int32_t(gap_blocks<DIM>(lo, hi, g, Dmin, nullptr) + (t < nS ? 1 : 0));
}

template <int DIM>
__global__ void k_gap_write(const uint64_t* __restrict__ S, const int64_t* __restrict__ d_nS,
                            int64_t ncap, KG g, int Dmin, const int64_t* __restrict__ offs,
                            uint64_t* __restrict__ out) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t > ncap) return;
  const int64_t nS = *d_nS;
  if (t > nS) return;
  uint64_t lo, hi;
  gap_bounds<DIM>(S, nS, t, g, &lo, &hi);
  int64_t o = offs[t];
  int64_t c = gap_blocks<DIM>(lo, hi, g, Dmin, out + o);
  if (t < nS) out[o + c] = S[t];
}

int read_bad(const int32_t* d_bad, bool* bad, cudaStream_t s, Err* err) {
  int32_t h = 0;
  FR_CUDA(err, cudaMemcpyAsync(&h, d_bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FR_CUDA(err, cudaStreamSynchronize(s));
  *bad = h != 0;
  return 0;
}

}  // namespace

#define DIM_DISPATCH(dim, ...)         \
  do {                                 \
    if ((dim) == 2) {                  \
      constexpr int D_ = 2;            \
      __VA_ARGS__;                     \
    } else {                           \
      constexpr int D_ = 3;            \
      __VA_ARGS__;                     \
    }                                  \
  } while (0)

int tree_encode(int dim, const KG& g, const int32_t* d_boxes, int64_t n, uint64_t* d_keys,
                cudaStream_t s, Err* err) {
  if (n <= 0) return 0;
  Alloc A{nullptr, s, err};
  Scratch S(&A);
  int32_t* bad = S.get<int32_t>(1);
  if (!bad) return set_error(err, FR_ENOMEM, "encode scratch");
  FR_CUDA(err, cudaMemsetAsync(bad, 0, 4, s));
  DIM_DISPATCH(dim, (k_encode<D_><<<nblk(n), TB, 0, s>>>(d_boxes, n, d_keys, g, bad)));
  FR_LAUNCH_CHECK(err);
  bool b = false;
  FR_TRY(read_bad(bad, &b, s, err));
  if (b) return set_error(err, FR_EINVAL, "box with depth/anchor out of range or misaligned");
  return 0;
}

int tree_complete(int dim, const KG& g, int Dmin, double L, const double* d_pts, int64_t n,
                  Buf<uint64_t>& out, int64_t* n_out, Alloc& A, cudaStream_t s, Err* err) {
  Scratch S(&A);
  int64_t nn = n > 0 ? n : 1;
  uint64_t* keys = S.get<uint64_t>(nn);
  uint64_t* tmp = S.get<uint64_t>(nn);
  uint64_t* seeds = S.get<uint64_t>(nn);
  int32_t* c1 = S.get<int32_t>(nn + 1);
  int64_t* o1 = S.get<int64_t>(nn + 1);
  int64_t* nS = S.get<int64_t>(1);
  int64_t* tot = S.get<int64_t>(1);
  if (!keys || !tmp || !seeds || !c1 || !o1 || !nS || !tot)
    return set_error(err, FR_ENOMEM, "completion scratch");
  if (n > 0) {
    DIM_DISPATCH(dim, (k_pts_encode<D_><<<nblk(n), TB, 0, s>>>(d_pts, n, L, g, keys)));
    FR_LAUNCH_CHECK(err);
    FR_TRY(radix_sort_keys(keys, tmp, n, dim * g.Dmax + g.mb, S, s, err));
    // unique seeds (all at depth Dmax, so linearisation only removes duplicates)
    DIM_DISPATCH(dim, (k_lin_count<D_><<<nblk(n), TB, 0, s>>>(keys, n, g, c1)));
    FR_LAUNCH_CHECK(err);
    FR_TRY(scan_counts(c1, o1, n, nS, S, s, err));
    k_compact<<<nblk(n), TB, 0, s>>>(keys, c1, o1, n, seeds);
    FR_LAUNCH_CHECK(err);
  } else {
    FR_CUDA(err, cudaMemsetAsync(nS, 0, 8, s));
  }
  int64_t ncap = n;  // gaps 0..nS with nS <= n
  DIM_DISPATCH(dim, (k_gap_count<D_><<<nblk(ncap + 1), TB, 0, s>>>(seeds, nS, ncap, g, Dmin, c1)));
  FR_LAUNCH_CHECK(err);
  FR_TRY(scan_counts(c1, o1, ncap + 1, tot, S, s, err));
  FR_TRY(read_i64(tot, n_out, s, err));
  FR_TRY(out.ensure(A, size_t(*n_out)));
  DIM_DISPATCH(dim, (k_gap_write<D_><<<nblk(ncap + 1), TB, 0, s>>>(seeds, nS, ncap, g, Dmin, o1, out.p)));
  FR_LAUNCH_CHECK(err);
  return 0;
}

int tree_uniform(int dim, const KG& g, int D, uint64_t* d_keys, cudaStream_t s, Err* err) {
  int64_t count = int64_t(1) << (dim * D);
  DIM_DISPATCH(dim, (k_uniform<D_><<<nblk(count), TB, 0, s>>>(d_keys, count, g, D)));
  FR_LAUNCH_CHECK(err);
  return 0;
}

int tree_linearise(int dim, const KG& g, uint64_t* d_keys, int64_t n, Buf<uint64_t>& out,
                   int64_t* n_out, Alloc& A, cudaStream_t s, Err* err) {
  Scratch S(&A);
  int32_t* cnt = S.get<int32_t>(n);
  int64_t* offs = S.get<int64_t>(n);
  int64_t* tot = S.get<int64_t>(1);
  if (!cnt || !offs || !tot) return set_error(err, FR_ENOMEM, "linearise scratch");
  if (n > 0) {
    DIM_DISPATCH(dim, (k_lin_count<D_><<<nblk(n), TB, 0, s>>>(d_keys, n, g, cnt)));
    FR_LAUNCH_CHECK(err);
  }
  FR_TRY(scan_counts(cnt, offs, n, tot, S, s, err));
  FR_TRY(read_i64(tot, n_out, s, err));
  FR_TRY(out.ensure(A, size_t(*n_out)));
  if (n > 0) {
    k_compact<<<nblk(n), TB, 0, s>>>(d_keys, cnt, offs, n, out.p);
    FR_LAUNCH_CHECK(err);
  }
  return 0;
}

// the write kernel adds up to this many tile totals per block (offs_base)
constexpr int64_t EDIT_SCAN_TILES_MAX = 256;

int tree_edit(int dim, const KG& g, int Dbase, const uint64_t* d_keys, const int8_t* d_flags,
              int64_t n, Buf<uint64_t>& out, int64_t* d_ctl, int32_t* d_bad, Alloc& A, cudaStream_t s,
              Err* err, Buf<int32_t>* org, Buf<int8_t>* otg, const KeyIndex& XO) {
  Scratch S(&A);
  int8_t* act = S.get<int8_t>(n);
  int32_t* cnt = S.get<int32_t>(n);
  int64_t* offs = S.get<int64_t>(n);
  if (!act || !cnt || !offs) return set_error(err, FR_ENOMEM, "edit scratch");
  // the edited tree has at most 2^dim leaves per old leaf: the output is sized for that bound and
  // the leaf count stays on the device for the balance passes
  FR_TRY(out.ensure(A, size_t(n) << dim));
  Offs O;
  const int64_t tiles = (n + SCAN_TILE_ITEMS - 1) / SCAN_TILE_ITEMS;
  if (tiles <= EDIT_SCAN_TILES_MAX) {
    // actions, counts and the tile-local scan in one launch; the write adds the tile bases
    int64_t* sums = S.get<int64_t>(tiles);
    if (!sums) return set_error(err, FR_ENOMEM, "edit scratch");
    DIM_DISPATCH(dim, (launch_dependent(k_edit_scan<D_>, unsigned(tiles), EDIT_SCAN_T, s, d_keys, d_flags, n, g, Dbase,
                                        act, offs, sums, d_ctl, d_bad)));
    FR_LAUNCH_CHECK(err);
    O = Offs{offs, sums, tiles, d_ctl + CTL_N};
  } else {
    DIM_DISPATCH(dim, (launch_dependent(k_edit_count<D_>, nblk(n), TB, s, d_keys, d_flags, n, g, Dbase, act, cnt,
                                        d_ctl, d_bad)));
    FR_LAUNCH_CHECK(err);
    FR_TRY(scan_counts_local(cnt, offs, n, d_ctl + CTL_N, S, s, err, &O));
  }
  if (org) {
    FR_TRY(org->ensure(A, size_t(n) << dim));
    FR_TRY(otg->ensure(A, size_t(n) << dim));
  }
  DIM_DISPATCH(dim, (launch_dependent(k_edit_write<D_>, nblk(n), TB, s, d_keys, act, O, n, g, out.p,
                                      reinterpret_cast<unsigned long long*>(d_ctl + CTL_REF),
                                      org ? org->p : nullptr, org ? otg->p : nullptr, XO)));
  FR_LAUNCH_CHECK(err);
  return 0;
}

// above this bound on the leaf count a pass first reads the exact count from the device
constexpr int64_t BAL_UB_MAX = int64_t(1) << 19;

static int read_ctl(const int64_t* d_ctl, int64_t* h_ctl, cudaStream_t s, Err* err) {
  if (cudaMemcpyAsync(h_ctl, d_ctl, CTL_SLOTS * sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return set_error(err, FR_ECUDA, "balance count read");
  return 0;
}

// one pass at depth D: count, scan, generate, sort, merge; octants beyond `cap` overflow the
// pass (small sort only).  `exact_G` >= 0: the host knows the generated count (sizes from it).
static int balance_pass(int dim, const KG& g, int D, Buf<uint64_t>& keys, Buf<uint64_t>& out,
                        Buf<uint64_t>& gen, Buf<uint64_t>& tmp, int64_t* d_ctl, int64_t n_ub,
                        int64_t exact_G, int64_t cap, const Offs& Ocnt, Alloc& A, cudaStream_t s,
                        Err* err, bool generated = false) {
  Scratch S(&A);
  const int64_t G_ub = exact_G >= 0 ? exact_G : cap;
  FR_TRY(out.ensure(A, size_t(n_ub + G_ub)));
  if (!generated) {  // otherwise gen already holds the pass's exact_G octants
    FR_TRY(gen.ensure(A, size_t(G_ub)));
    DIM_DISPATCH(dim, (launch_dependent(k_bal_gen<D_>, nblk(n_ub * BalLanes<D_>::value), TB, s, keys.p, d_ctl, n_ub, g, D,
                                        Ocnt, gen.p, cap)));
    FR_LAUNCH_CHECK(err);
  }
  if (exact_G < 0 || exact_G <= SMALL_SORT_MAX) {
    launch_dependent(k_sort_small, 1, 1024, s, gen.p, d_ctl, cap, D);
    FR_LAUNCH_CHECK(err);
  } else {
    FR_TRY(tmp.ensure(A, size_t(exact_G)));
    FR_TRY(radix_sort_keys(gen.p, tmp.p, exact_G, dim * g.Dmax + g.mb, S, s, err));
  }
  // with exact sizes (large sets, which carry many duplicate requests) the generated octants are
  // linearised in parallel first, their count replacing ctl[CTL_G]; small sets are linearised
  // inside the merge, range by range
  const bool lin_first = exact_G >= 0;
  const uint64_t* src = gen.p;
  if (lin_first) {
    int32_t* cl = S.get<int32_t>(exact_G);
    int64_t* ol = S.get<int64_t>(exact_G);
    if (!cl || !ol) return set_error(err, FR_ENOMEM, "balance linearise scratch");
    FR_TRY(tmp.ensure(A, size_t(exact_G)));
    DIM_DISPATCH(dim, (k_lin_count<D_><<<nblk(exact_G), TB, 0, s>>>(gen.p, exact_G, g, cl)));
    FR_LAUNCH_CHECK(err);
    FR_TRY(scan_counts(cl, ol, exact_G, d_ctl + CTL_G, S, s, err));
    k_compact<<<nblk(exact_G), TB, 0, s>>>(gen.p, cl, ol, exact_G, tmp.p);
    FR_LAUNCH_CHECK(err);
    src = tmp.p;
  }
  int32_t* cnt2 = S.get<int32_t>(n_ub);
  int64_t* lo = S.get<int64_t>(n_ub);
  int64_t* offs2 = S.get<int64_t>(n_ub);
  if (!cnt2 || !lo || !offs2) return set_error(err, FR_ENOMEM, "balance merge scratch");
  DIM_DISPATCH(dim, (launch_dependent(k_merge_count<D_>, nblk(n_ub), TB, s, keys.p, d_ctl, n_ub, src, cap, g,
                                      lin_first, cnt2, lo)));
  FR_LAUNCH_CHECK(err);
  // the merged tree has at most n + G leaves; its count replaces ctl[CTL_N] on the device
  Offs Om;
  FR_TRY(scan_counts_local(cnt2, offs2, n_ub, d_ctl + CTL_N, S, s, err, &Om));
  DIM_DISPATCH(dim, (launch_dependent(k_merge_write<D_>, nblk(n_ub), TB, s, keys.p, d_ctl, n_ub, src, cap, g,
                                      lin_first, cnt2, lo, Om, out.p)));
  FR_LAUNCH_CHECK(err);
  Buf<uint64_t> t = keys;  // the merged tree becomes the tree
  keys = out;
  out = t;
  return 0;
}

int tree_balance(int dim, const KG& g, int Dhigh, int Dlow, Buf<uint64_t>& keys, int64_t* d_ctl,
                 int64_t n_ub, int64_t* h_ctl, Alloc& A, cudaStream_t s, Err* err) {
  Buf<uint64_t> gen, tmp, out;
  int rc = 0;
  bool known = false;  // h_ctl holds the current control block
  for (int D = Dhigh; D >= Dlow && D >= 2; --D) {
    if (!known && n_ub > BAL_UB_MAX) {
      // large trees: generating up to a loose bound costs more than a synchronisation
      if ((rc = read_ctl(d_ctl, h_ctl, s, err))) break;
      n_ub = h_ctl[CTL_N];
    }
    Scratch S(&A);
    // one search pass: the octants are placed by an atomic counter (sorted next, so their order
    // does not matter) into room for max(2^16, 2n) of them; a pass that generates more is counted,
    // scanned and generated again at exact positions
    const int64_t capG = 2 * n_ub > (int64_t(1) << 16) ? 2 * n_ub : (int64_t(1) << 16);
    if (gen.ensure(A, size_t(capG)) || cudaMemsetAsync(d_ctl + CTL_G, 0, 8, s) != cudaSuccess) {
      rc = set_error(err, FR_ENOMEM, "balance scratch");
      break;
    }
    DIM_DISPATCH(dim, (launch_dependent(k_bal_gen_fast<D_>, nblk(n_ub * BalLanes<D_>::value), TB, s, keys.p, d_ctl,
                                        n_ub, g, D, gen.p, capG, false, int(CTL_N), int(CTL_G), KeyIndex{})));
    ++launch_counter();
    if ((rc = cudaGetLastError() != cudaSuccess ? set_error(err, FR_ECUDA, "k_bal_gen_fast") : 0)) break;
    // the pass's one synchronisation: leaf count, generated count (and the edit's statistics)
    if ((rc = read_ctl(d_ctl, h_ctl, s, err))) break;
    known = true;
    const int64_t n = h_ctl[CTL_N];
    int64_t G = h_ctl[CTL_G];
    n_ub = n;
    if (G == 0) continue;
    if (G <= capG) {
      rc = balance_pass(dim, g, D, keys, out, gen, tmp, d_ctl, n, G, G, Offs{}, A, s, err, true);
    } else {
      // the exact count (every lane's octants, duplicates included) sizes the regeneration
      int32_t* cnt = S.get<int32_t>(n);
      int64_t* offs = S.get<int64_t>(n);
      if (!cnt || !offs) {
        rc = set_error(err, FR_ENOMEM, "balance scratch");
        break;
      }
      DIM_DISPATCH(dim, (launch_dependent(k_bal_count<D_>, nblk(n * BalLanes<D_>::value), TB, s, keys.p, d_ctl, n, g, D, cnt)));
      ++launch_counter();
      if ((rc = cudaGetLastError() != cudaSuccess ? set_error(err, FR_ECUDA, "k_bal_count") : 0)) break;
      if ((rc = scan_counts(cnt, offs, n, d_ctl + CTL_G, S, s, err))) break;
      if ((rc = read_ctl(d_ctl, h_ctl, s, err))) break;
      G = h_ctl[CTL_G];
      rc = balance_pass(dim, g, D, keys, out, gen, tmp, d_ctl, n, G, G, Offs{offs, nullptr, 0, d_ctl + CTL_G}, A, s,
                        err);
    }
    if (rc) break;
    n_ub = n + G;
    known = false;
  }
  if (!rc && !known) rc = read_ctl(d_ctl, h_ctl, s, err);
  gen.release(A);
  tmp.release(A);
  out.release(A);
  return rc;
}

int tree_balance_async(int dim, const KG& g, int Dlow, Buf<uint64_t>& keys, int64_t* d_ctl,
                       int64_t* n_ub, Alloc& A, cudaStream_t s, Err* err, Buf<int32_t>* org,
                       Buf<int8_t>* otg, int* n_slot, KeyIndex* X, uint64_t* spare_tab) {
  Buf<uint64_t> gen, out;
  Buf<int32_t> org_out;
  Buf<int8_t> otg_out;
  int rc = 0;
  const int64_t cap = SMALL_SORT_MAX;
  int passes = 0;
  for (int D = g.Dmax; D >= Dlow && D >= 2; --D) ++passes;
  // key bits and the containing leaf's index fit one 64-bit value, on every pass: then each
  // pass's merge sorts the octants itself (k_merge_sorted), otherwise a one-block kernel sorts
  // them and computes the shifts (k_sort_annot)
  const bool packed = dim * g.Dmax + g.mb + PACK_BITS <= 64 &&
                      *n_ub + int64_t(passes) * cap < (int64_t(1) << PACK_BITS);
  // the key index travels with the tree only through passes that write it (k_merge_sorted)
  if (!packed || !spare_tab) X->tab = nullptr;
  int grid_cap = 0;
  if (packed) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return set_error(err, FR_ECUDA, "device attribute");
    grid_cap = 2 * sms;  // two resident 1024-thread blocks per SM: one wave
  }
  // leaf-count slots: pass k reads sn and writes the next one (packed: CTL_N -> NB -> NA -> NB ...,
  // otherwise CTL_N throughout); octant counters alternate between CTL_G and CTL_GB
  int sn = CTL_N;
  for (int D = g.Dmax, kp = 0; D >= Dlow && D >= 2; --D, ++kp) {
    Scratch S(&A);
    const int64_t nb = *n_ub;
    const int sg = (packed && (kp & 1)) ? CTL_GB : CTL_G;
    int32_t* P = packed ? nullptr : S.get<int32_t>(cap + 1);
    if ((!packed && !P) || gen.ensure(A, size_t(cap)) || out.ensure(A, size_t(nb + cap)) ||
        (org && (org_out.ensure(A, size_t(nb + cap)) || otg_out.ensure(A, size_t(nb + cap))))) {
      rc = set_error(err, FR_ENOMEM, "balance scratch");
      break;
    }
    DIM_DISPATCH(dim, (launch_dependent(k_bal_gen_fast<D_>, nblk(nb * BalLanes<D_>::value), TB, s, keys.p, d_ctl, nb, g,
                                        D, gen.p, cap, packed, sn, sg, *X)));
    ++launch_counter();
    if (packed) {
      const int so = (kp & 1) ? CTL_NA : CTL_NB;
      const int sg_next = (kp & 1) ? CTL_G : CTL_GB;
      int64_t grid = nblk(nb, 1024);
      if (grid > grid_cap) grid = grid_cap;
      DIM_DISPATCH(dim, (launch_dependent(k_merge_sorted<D_>, unsigned(grid), 1024, s, static_cast<const uint64_t*>(keys.p),
                                          d_ctl, nb, static_cast<const uint64_t*>(gen.p), cap, D, sn, sg, so,
                                          sg_next, g, out.p, static_cast<const int32_t*>(org ? org->p : nullptr),
                                          static_cast<const int8_t*>(org ? otg->p : nullptr),
                                          org ? org_out.p : nullptr, org ? otg_out.p : nullptr,
                                          KeyIndex{X->tab ? spare_tab : nullptr, X->sh})));
      ++launch_counter();
      sn = so;
      if (X->tab) std::swap(X->tab, spare_tab);
    } else {
      DIM_DISPATCH(dim, (launch_dependent(k_sort_annot<D_>, 1, 1024, s, gen.p, d_ctl, cap, D,
                                          static_cast<const uint64_t*>(keys.p), g, P, packed)));
      ++launch_counter();
      DIM_DISPATCH(dim, (launch_dependent(k_merge_fast<D_>, nblk(nb), TB, s, static_cast<const uint64_t*>(keys.p),
                                          static_cast<const int64_t*>(d_ctl), nb, static_cast<const uint64_t*>(gen.p),
                                          static_cast<const int32_t*>(P), g, out.p,
                                          static_cast<const int32_t*>(org ? org->p : nullptr),
                                          static_cast<const int8_t*>(org ? otg->p : nullptr),
                                          org ? org_out.p : nullptr, org ? otg_out.p : nullptr)));
      ++launch_counter();
    }
    if (cudaGetLastError() != cudaSuccess) {
      rc = set_error(err, FR_ECUDA, "balance pass launch");
      break;
    }
    Buf<uint64_t> t = keys;  // the merged tree becomes the tree
    keys = out;
    out = t;
    if (org) {
      std::swap(*org, org_out);
      std::swap(*otg, otg_out);
    }
    *n_ub = nb + cap;
  }
  *n_slot = sn;
  gen.release(A);
  out.release(A);
  org_out.release(A);
  otg_out.release(A);
  return rc;
}

int tree_map(int dim, const KG& g, const uint64_t* d_old, int64_t n_old, const uint64_t* d_new,
             int64_t n_new, const int64_t* d_n_new, int32_t* d_src, int8_t* d_tag, int32_t* d_bad,
             cudaStream_t s, Err* err) {
  if (n_new <= 0) return 0;
  DIM_DISPATCH(dim, (launch_dependent(k_map<D_>, nblk(n_new), TB, s, d_old, n_old, d_new, n_new, d_n_new, g, d_src, d_tag, d_bad)));
  FR_LAUNCH_CHECK(err);
  return 0;
}
int tree_conn(int dim, const KG& g, const uint64_t* d_keys, int64_t n, const int64_t* d_n, int32_t* d_nbr,
              int8_t* d_ftype, int8_t* d_slot, int32_t* d_contrib, int32_t* d_bad, cudaStream_t s,
              Err* err, int64_t* d_fcnt, const FaceLists& L) {
  if (n <= 0) return 0;
  const int64_t T = n * 2 * dim;
  // blocks of whole leaves: 64 leaves (2D, 256 threads) or 32 (3D, 192 threads)
  const int bt = dim == 2 ? 256 : 192;
  DIM_DISPATCH(dim, (launch_dependent(k_conn<D_>, nblk(T, bt), bt, s, d_keys, n, d_n, g, d_nbr, d_ftype, d_slot,
                                      d_contrib, d_bad, d_fcnt, L)));
  FR_LAUNCH_CHECK(err);
  return 0;
}

int tree_validate_async(int dim, const KG& g, const uint64_t* d_keys, int64_t n, int Dlo, int Dhi,
                        int32_t* d_bad, cudaStream_t s, Err* err) {
  if (n <= 0) return 0;
  DIM_DISPATCH(dim, (k_validate<D_><<<nblk(n), TB, 0, s>>>(d_keys, n, g, Dlo, Dhi, d_bad)));
  FR_LAUNCH_CHECK(err);
  return 0;
}

int tree_validate(int dim, const KG& g, const uint64_t* d_keys, int64_t n, int Dlo, int Dhi,
                  bool* ok, Alloc& A, cudaStream_t s, Err* err) {
  Scratch S(&A);
  int32_t* bad = S.get<int32_t>(1);
  if (!bad) return set_error(err, FR_ENOMEM, "validate scratch");
  FR_CUDA(err, cudaMemsetAsync(bad, 0, 4, s));
  if (n > 0) {
    DIM_DISPATCH(dim, (k_validate<D_><<<nblk(n), TB, 0, s>>>(d_keys, n, g, Dlo, Dhi, bad)));
    FR_LAUNCH_CHECK(err);
  }
  bool b = true;
  FR_TRY(read_bad(bad, &b, s, err));
  *ok = !b && n > 0;
  return 0;
}

}  // namespace frg
