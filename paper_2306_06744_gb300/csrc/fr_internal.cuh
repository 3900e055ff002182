// fr_internal.cuh -- internal declarations of the GB300 adaptive-FR library.
// Key arithmetic (Sec. 2.2), device buffers, operator tables and the primitive entry points
// (scan, radix sort, binary search) shared by the tree and solver translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "fr.h"

namespace frg {

// ---------------------------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------------------------
struct Err {
  int code = 0;
  std::string msg;
};
int set_error(Err* e, int code, const std::string& msg);
Err* global_err();

#define FR_TRY(expr)          \
  do {                        \
    int rc_ = (expr);         \
    if (rc_ != 0) return rc_; \
  } while (0)

#define FR_CUDA(err, expr)                                                                   \
  do {                                                                                       \
    cudaError_t ce_ = (expr);                                                                \
    if (ce_ != cudaSuccess)                                                                  \
      return ::frg::set_error((err), FR_ECUDA,                                               \
                              std::string(#expr) + ": " + cudaGetErrorString(ce_));          \
  } while (0)

// every kernel launch is followed by this check, which also counts the launch
int64_t& launch_counter();
#define FR_LAUNCH_CHECK(err)            \
  do {                                  \
    ++::frg::launch_counter();          \
    FR_CUDA(err, cudaGetLastError());   \
  } while (0)

// Programmatic dependent launch: the time-step and adaptation kernels are launched so that their
// blocks may be scheduled while the predecessor in the stream drains.  Every such kernel first
// waits (in hardware) until the predecessor grid has completed and its writes are visible, and
// only then lets its own dependents launch, so a kernel never overlaps anything but the tail of
// its immediate predecessor, and all its reads and writes come after that wait.  (Without the
// launch attribute the wait returns at once.)
__device__ __forceinline__ void pdl_wait_then_release() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
// Reads issued before pdl_wait_then_release may only touch data final before the predecessor
// started (its own predecessor's outputs, or static tables): a kernel releases its dependents only
// after its own wait, so when a kernel starts early, everything but its immediate predecessor has
// completed.  Writes always come after the wait.

template <class Kern, class... Args>
cudaError_t launch_dependent(Kern kernel, unsigned grid, unsigned block, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// launch_dependent with dynamic shared memory (see residency_pad)
template <class Kern, class... Args>
cudaError_t launch_dependent_smem(Kern kernel, unsigned grid, unsigned block, size_t dyn_smem,
                                  cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = dyn_smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Unused dynamic shared memory that holds a kernel to at most max_warps resident warps per SM:
// the smallest per-block footprint that no longer fits one block more than that; 0 where shared
// memory already allows no more (or the attributes cannot be read).
template <class Kern>
size_t residency_pad(Kern kernel, int threads, int max_warps) {
  cudaFuncAttributes fa;
  int dev = 0, smem_sm = 0, reserved = 0;
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int blocks = max_warps / ((threads + 31) / 32);
  if (blocks < 1) return 0;
  const long need = long(smem_sm) / (blocks + 1) + 1;  // footprint above which blocks+1 do not fit
  long pad = need - long(reserved) - long(fa.sharedSizeBytes);
  if (pad <= 0) return 0;
  pad = (pad + 127) / 128 * 128;
  if (long(reserved) + long(fa.sharedSizeBytes) + pad > long(smem_sm) / blocks) return 0;
  return size_t(pad);
}

// ---------------------------------------------------------------------------------------------
// Morton IDs (Sec. 2.2, Algorithm 1).  Bits are interleaved with the "magic number" bit spread
// the paper mentions: spreading one coordinate's bits to every dim-th position by masked shifts.
// The full-resolution interleave of an anchor whose low Dmax-D bits are zero equals the paper's
// interleave of the depth-D coordinate followed by dim*(Dmax-D) zero bits.
// ---------------------------------------------------------------------------------------------
struct KeyGeo {
  int dim, Dmax, mb;
};

inline int depth_bits(int Dmax) {
  int mb = 0;
  while ((1 << mb) < Dmax + 1) ++mb;
  return mb;
}

__host__ __device__ __forceinline__ uint64_t spread2(uint64_t x) {
  x &= 0xFFFFFFFFull;
  x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
  x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}
__host__ __device__ __forceinline__ uint64_t compact2(uint64_t x) {
  x &= 0x5555555555555555ull;
  x = (x ^ (x >> 1)) & 0x3333333333333333ull;
  x = (x ^ (x >> 2)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x ^ (x >> 4)) & 0x00FF00FF00FF00FFull;
  x = (x ^ (x >> 8)) & 0x0000FFFF0000FFFFull;
  x = (x ^ (x >> 16)) & 0x00000000FFFFFFFFull;
  return x;
}
__host__ __device__ __forceinline__ uint64_t spread3(uint64_t x) {
  x &= 0x1FFFFFull;
  x = (x | (x << 32)) & 0x001F00000000FFFFull;
  x = (x | (x << 16)) & 0x001F0000FF0000FFull;
  x = (x | (x << 8)) & 0x100F00F00F00F00Full;
  x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}
__host__ __device__ __forceinline__ uint64_t compact3(uint64_t x) {
  x &= 0x1249249249249249ull;
  x = (x ^ (x >> 2)) & 0x10C30C30C30C30C3ull;
  x = (x ^ (x >> 4)) & 0x100F00F00F00F00Full;
  x = (x ^ (x >> 8)) & 0x001F0000FF0000FFull;
  x = (x ^ (x >> 16)) & 0x001F00000000FFFFull;
  x = (x ^ (x >> 32)) & 0x00000000001FFFFFull;
  return x;
}

template <int DIM>
__host__ __device__ __forceinline__ uint64_t interleave(const uint32_t* x) {
  if (DIM == 2) return spread2(x[0]) | (spread2(x[1]) << 1);
  return spread3(x[0]) | (spread3(x[1]) << 1) | (spread3(x[2]) << 2);
}
template <int DIM>
__host__ __device__ __forceinline__ void deinterleave(uint64_t raw, uint32_t* x) {
  if (DIM == 2) {
    x[0] = uint32_t(compact2(raw));
    x[1] = uint32_t(compact2(raw >> 1));
  } else {
    x[0] = uint32_t(compact3(raw));
    x[1] = uint32_t(compact3(raw >> 1));
    x[2] = uint32_t(compact3(raw >> 2));
  }
}

// Device-side view of the key layout.
struct KG {
  int Dmax, mb;
  __host__ __device__ __forceinline__ int depth(uint64_t k) const { return int(k & ((1ull << mb) - 1)); }
  __host__ __device__ __forceinline__ uint64_t raw(uint64_t k) const { return k >> mb; }
  __host__ __device__ __forceinline__ uint64_t make(uint64_t raw, int d) const { return (raw << mb) | uint64_t(d); }
  __host__ __device__ __forceinline__ uint32_t width(int d) const { return 1u << (Dmax - d); }
};

template <int DIM>
__host__ __device__ __forceinline__ uint64_t vol_raw(const KG& g, int d) {
  return 1ull << (DIM * (g.Dmax - d));  // raw-ID span of one octant at depth d
}
template <int DIM>
__host__ __device__ __forceinline__ uint64_t key_end(const KG& g, uint64_t k) {
  // smallest key beyond the subtree of k (every descendant of k is below it)
  return (g.raw(k) + vol_raw<DIM>(g, g.depth(k))) << g.mb;
}
template <int DIM>
__host__ __device__ __forceinline__ bool is_ancestor(const KG& g, uint64_t a, uint64_t b) {
  return b > a && b < key_end<DIM>(g, a);
}
template <int DIM>
__host__ __device__ __forceinline__ uint64_t child_key(const KG& g, uint64_t k, int c) {
  int d = g.depth(k);
  return g.make(g.raw(k) + uint64_t(c) * vol_raw<DIM>(g, d + 1), d + 1);
}
template <int DIM>
__host__ __device__ __forceinline__ uint64_t parent_key(const KG& g, uint64_t k) {
  int d = g.depth(k);
  uint64_t span = vol_raw<DIM>(g, d - 1);
  return g.make(g.raw(k) / span * span, d - 1);
}
template <int DIM>
__host__ __device__ __forceinline__ int child_index(const KG& g, uint64_t k) {
  int d = g.depth(k);
  return int((g.raw(k) >> (DIM * (g.Dmax - d))) & ((1u << DIM) - 1));
}
// key of the finest cell at integer point x (point location queries)
template <int DIM>
__host__ __device__ __forceinline__ uint64_t cell_key(const KG& g, const uint32_t* x) {
  return g.make(interleave<DIM>(x), g.Dmax);
}

// first index in a[0..n) with a[i] >= v / > v
__device__ __forceinline__ int64_t lower_bound_dev(const uint64_t* a, int64_t n, uint64_t v) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (__ldg(a + mid) < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ int64_t upper_bound_dev(const uint64_t* a, int64_t n, uint64_t v) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (__ldg(a + mid) <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Sampled index of a sorted key array k[0..n): tab[j] = k[j << sh] for j < ceil(n / 2^sh),
// written by the kernel that writes k (KeyIndex::note at every output position).  A search first
// bisects the samples, staged in shared memory, then the 2^sh keys between two samples: on a tree
// of 20k leaves and sh = 7 that is about 4 dependent global reads instead of 15.
constexpr int KEY_INDEX_MAX = 1024;  // samples per index (8 KB of shared memory)
struct KeyIndex {
  uint64_t* tab = nullptr;  // null: no index (a plain binary search)
  int sh = 0;
  __device__ __forceinline__ void note(int64_t o, uint64_t key) const {
    if (tab && (o & ((int64_t(1) << sh) - 1)) == 0) tab[o >> sh] = key;
  }
};
// the smallest sampling shift >= 7 that keeps an index of n_ub keys within KEY_INDEX_MAX samples
inline int key_index_shift(int64_t n_ub) {
  int sh = 7;
  while (((n_ub + (int64_t(1) << sh) - 1) >> sh) > KEY_INDEX_MAX) ++sh;
  return sh;
}
// Block-wide (every thread calls it): stages the samples of an index of n keys in s_tab and
// returns their count (0 without an index).  Ends with a block barrier.
__device__ __forceinline__ int stage_key_index(const KeyIndex& X, int64_t n, uint64_t* s_tab) {
  const int m = X.tab ? int((n + (int64_t(1) << X.sh) - 1) >> X.sh) : 0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) s_tab[j] = X.tab[j];
  __syncthreads();
  return m;
}
// first index in k[0..n) with k[i] > v (upper) or >= v (lower), using m staged samples
// (m = 0: plain binary search)
template <bool UPPER>
__device__ __forceinline__ int64_t bound_indexed(const uint64_t* k, int64_t n, uint64_t v, const uint64_t* s_tab,
                                                 int m, int sh) {
  int64_t a = 0, b = n;
  if (m > 0) {
    int lo = 0, hi = m;  // first sample past v
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (UPPER ? (s_tab[mid] <= v) : (s_tab[mid] < v)) lo = mid + 1; else hi = mid;
    }
    if (lo == 0) return 0;  // k[0] is the first sample
    // k[(lo-1) << sh] is before the bound, and k[lo << sh] (if any) is past it
    a = (int64_t(lo - 1) << sh) + 1;
    b = int64_t(lo) << sh;
    if (b > n) b = n;
  }
  while (a < b) {
    const int64_t mid = (a + b) >> 1;
    const uint64_t x = __ldg(k + mid);
    if (UPPER ? (x <= v) : (x < v)) a = mid + 1; else b = mid;
  }
  return a;
}

// Old->new mapping of one new leaf (Sec. 4.2, mapping algorithm) by one lower bound in the old
// keys: tag 0 copy of old leaf *src, 1 refined from old leaf *src, 2 fused from the 2^dim old
// leaves starting at *src.  A new leaf that is none of these makes the tree pair invalid: *bad is
// set and an in-bounds copy is emitted so later kernels stay in bounds.
template <int DIM>
__device__ __forceinline__ void map_leaf(const uint64_t* __restrict__ old, int64_t no, uint64_t key, const KG& g,
                                         int32_t* src, int8_t* tag, int32_t* bad) {
  const int64_t B = lower_bound_dev(old, no, key);
  if (B < no && old[B] == key) {
    *src = int32_t(B);
    *tag = 0;
  } else if (B > 0 && is_ancestor<DIM>(g, old[B - 1], key)) {
    *src = int32_t(B - 1);
    *tag = 1;
  } else {
    bool ok = B + (1 << DIM) <= no;
    for (int c = 0; c < (1 << DIM) && ok; ++c) ok = old[B + c] == child_key<DIM>(g, key, c);
    if (ok) {
      *src = int32_t(B);
      *tag = 2;
    } else {
      atomicExch(bad, 1);
      *src = int32_t(B < no ? B : no - 1);
      *tag = 0;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Device memory: caller allocator or stream-ordered cudaMallocAsync.
// ---------------------------------------------------------------------------------------------
// Blocks released by a mesh are kept for reuse on the same stream (stream order makes the reuse
// safe) instead of going back to the caller's allocator every time; they are returned at
// fr_mesh_free.
struct BlockCache {
  std::vector<std::pair<void*, size_t>> free_blocks;
  std::vector<std::pair<void*, size_t>> live;  // block -> size of blocks handed out
};

struct Alloc {
  const fr_allocator* user = nullptr;
  cudaStream_t stream = nullptr;
  Err* err = nullptr;
  BlockCache* cache = nullptr;
  void* get(size_t bytes);
  void put(void* p);
  void release_cache();
};

template <class T>
struct Buf {
  T* p = nullptr;
  size_t cap = 0;
  // grows (never shrinks) to hold n elements; contents are not preserved
  int ensure(Alloc& A, size_t n, double slack = 1.25) {
    if (n <= cap && p) return 0;
    if (p) A.put(p);
    p = nullptr;
    cap = 0;
    size_t want = size_t(double(n) * slack) + 16;
    p = static_cast<T*>(A.get(want * sizeof(T)));
    if (!p) return set_error(A.err, FR_ENOMEM, "device allocation failed");
    cap = want;
    return 0;
  }
  void release(Alloc& A) {
    if (p) A.put(p);
    p = nullptr;
    cap = 0;
  }
};

// scratch buffers released at scope exit (stream-ordered, so safe with pending kernels)
struct Scratch {
  Alloc* A;
  std::vector<void*> ptrs;
  explicit Scratch(Alloc* a) : A(a) {}
  ~Scratch() {
    for (void* p : ptrs) A->put(p);
  }
  template <class T>
  T* get(size_t n) {
    void* p = A->get((n ? n : 1) * sizeof(T));
    if (p) ptrs.push_back(p);
    return static_cast<T*>(p);
  }
};

// ---------------------------------------------------------------------------------------------
// Primitives (fr_prim.cu)
// ---------------------------------------------------------------------------------------------
// exclusive scan of int32 counts into int64 offsets; the total goes to *d_total (device)
// Exclusive offsets produced by a scan: global (sums == nullptr, total already stored), or local
// to tiles of SCAN_TILE_ITEMS items with the tile totals in sums[nb]; a consumer kernel then adds
// its tile's base itself (offs_base) and its block 0 stores the grand total to *total, which saves
// the scan's second launch.
constexpr int64_t SCAN_TILE_ITEMS = 2048;
struct Offs {
  const int64_t* offs;
  const int64_t* sums;
  int64_t nb;
  int64_t* total;
};
// Block-wide (every thread of the block calls it; blockDim a power of two <= 256; the block's
// items, the first of which is i0, lie in one tile): the base of the block's tile, and the grand
// total in *grand; block 0 stores the total.
__device__ __forceinline__ int64_t offs_base(const Offs& O, int64_t i0, int64_t* grand) {
  __shared__ int64_t red[256];
  if (!O.sums) {
    *grand = 0;
    return 0;
  }
  const int t = threadIdx.x, nt = blockDim.x;
  const int64_t tile = i0 / SCAN_TILE_ITEMS;
  int64_t a = 0, b = 0;
  for (int64_t k = t; k < O.nb; k += nt) {
    const int64_t v = O.sums[k];
    b += v;
    if (k < tile) a += v;
  }
  red[t] = a;
  __syncthreads();
  for (int st = nt / 2; st > 0; st >>= 1) {
    if (t < st) red[t] += red[t + st];
    __syncthreads();
  }
  const int64_t base = red[0];
  __syncthreads();
  red[t] = b;
  __syncthreads();
  for (int st = nt / 2; st > 0; st >>= 1) {
    if (t < st) red[t] += red[t + st];
    __syncthreads();
  }
  *grand = red[0];
  if (blockIdx.x == 0 && t == 0) *O.total = red[0];
  __syncthreads();
  return base;
}
// scan whose second pass is left to the consumer when the input spans at most 256 tiles
int scan_counts_local(const int32_t* d_in, int64_t* d_out, int64_t n, int64_t* d_total, Scratch& S,
                      cudaStream_t s, Err* err, Offs* O);
int scan_counts64_local(const int64_t* d_in, int64_t* d_out, int64_t n, int64_t* d_total, Scratch& S,
                        cudaStream_t s, Err* err, Offs* O);
int scan_counts(const int32_t* d_in, int64_t* d_out, int64_t n, int64_t* d_total, Scratch& S,
                cudaStream_t s, Err* err);
int scan_counts64(const int64_t* d_in, int64_t* d_out, int64_t n, int64_t* d_total, Scratch& S,
                  cudaStream_t s, Err* err);
// ascending LSD radix sort of n keys over the low `bits` bits; d_tmp holds n keys of scratch
int radix_sort_keys(uint64_t* d_keys, uint64_t* d_tmp, int64_t n, int bits, Scratch& S,
                    cudaStream_t s, Err* err);
// reads a device int64 to the host (synchronises the stream)
int read_i64(const int64_t* d, int64_t* h, cudaStream_t s, Err* err);

// ---------------------------------------------------------------------------------------------
// Tree pipeline (fr_tree.cu), on device arrays
// ---------------------------------------------------------------------------------------------
struct TreeOut {
  Buf<uint64_t>* keys;  // output tree (grown as needed)
  int64_t n;
};
int tree_encode(int dim, const KG& g, const int32_t* d_boxes, int64_t n, uint64_t* d_keys,
                cudaStream_t s, Err* err);
int tree_uniform(int dim, const KG& g, int D, uint64_t* d_keys, cudaStream_t s, Err* err);
int tree_complete(int dim, const KG& g, int Dmin, double L, const double* d_pts, int64_t n,
                  Buf<uint64_t>& out, int64_t* n_out, Alloc& A, cudaStream_t s, Err* err);
int tree_linearise(int dim, const KG& g, uint64_t* d_keys_sorted, int64_t n, Buf<uint64_t>& out,
                   int64_t* n_out, Alloc& A, cudaStream_t s, Err* err);
// Control block of an adaptation on the device, CTL_SLOTS int64 values (layout in fr_tree.cu):
// [0] leaf count of the tree being built, [1] generated octants of the current balance pass,
// [2] refined leaves, [3] coarsened groups, [4] overflowed pass depth (0: none), [5] passes that
// changed the tree, [6] face-list counts (conforming | hanging << 32); for the merge of a balance
// pass issued without synchronisation: [7] the leaf count before the pass, [8] the sorted
// octants it merges; [9] blocks of the connectivity kernel that have finished (FaceLists::pub);
// for balance passes whose merge sorts the octants itself (tree_balance_async): [10], [11] the
// leaf counts the passes hand on (alternately), [12] the second generated-octant counter.
enum {
  CTL_N = 0, CTL_G = 1, CTL_REF = 2, CTL_COARSE = 3, CTL_OVER = 4, CTL_PASSES = 5, CTL_FACES = 6,
  CTL_NPREV = 7, CTL_GS = 8, CTL_DONE = 9, CTL_NA = 10, CTL_NB = 11, CTL_GB = 12, CTL_SLOTS = 13
};
// The edit zeroes the control block (and the two error flags d_bad, if given) and leaves its
// leaf count and statistics there without a host synchronisation; its output holds at most
// n << dim leaves.  With org/otg: each edited leaf's origin in the old tree and its relation to
// it (0 the same leaf, 1 inside it, 2 the parent of the 2^dim old leaves from the origin on).
int tree_edit(int dim, const KG& g, int Dbase, const uint64_t* d_keys, const int8_t* d_flags,
              int64_t n, Buf<uint64_t>& out, int64_t* d_ctl, int32_t* d_bad, Alloc& A, cudaStream_t s,
              Err* err, Buf<int32_t>* org = nullptr, Buf<int8_t>* otg = nullptr,
              const KeyIndex& XO = KeyIndex{});
// balances `keys` in place for depth passes D = Dhigh .. Dlow with exact sizes (one host
// synchronisation per pass); the leaf count is d_ctl[0] on entry (at most n_ub) and h_ctl
// (CTL_SLOTS values) holds the final control block on return
int tree_balance(int dim, const KG& g, int Dhigh, int Dlow, Buf<uint64_t>& keys, int64_t* d_ctl,
                 int64_t n_ub, int64_t* h_ctl, Alloc& A, cudaStream_t s, Err* err);
// the same passes (Dmax .. Dlow) issued without any host synchronisation: each pass may generate
// at most 4096 octants, *n_ub is raised to a bound of the final leaf count, and a pass that would
// generate more sets d_ctl[4] to its depth and leaves the tree unchanged from there on (the caller
// then finishes with tree_balance from that depth).  With org/otg (those of the edit): carried
// through the passes, so that they give every leaf of the balanced tree its origin in the tree
// before the edit and its relation to it, as the old->new mapping (tree_map) would.  *n_slot
// receives the control-block slot that holds the balanced tree's leaf count (CTL_N, or one of the
// slots the passes hand the count on in).
// X (in/out): the index of keys (tab null: none), carried through the passes that sort their
// octants themselves, with spare_tab (as large as X's table) as the other buffer; on return the
// index of the balanced tree, or none.
int tree_balance_async(int dim, const KG& g, int Dlow, Buf<uint64_t>& keys, int64_t* d_ctl,
                       int64_t* n_ub, Alloc& A, cudaStream_t s, Err* err, Buf<int32_t>* org,
                       Buf<int8_t>* otg, int* n_slot, KeyIndex* X, uint64_t* spare_tab);
// d_n_new / d_n (nullable): device leaf count of the new tree; n_new / n is then an upper bound
int tree_map(int dim, const KG& g, const uint64_t* d_old, int64_t n_old, const uint64_t* d_new,
             int64_t n_new, const int64_t* d_n_new, int32_t* d_src, int8_t* d_tag, int32_t* d_bad,
             cudaStream_t s, Err* err);
// connectivity; d_contrib (may be null) receives [n][2dim][4] coarse-side contributors
// d_fcnt (nullable): per leaf (n entries) the face-list counts, conforming faces owned (the + faces
// of conforming pairs) in the low 32 bits and coarse sides of hanging faces in the high 32 bits;
// zero past the device count
// L (conf null: off): the face lists written by the connectivity kernel itself, each block's
// faces appended at a base taken from *L.count (conforming count low 32 bits, hanging high), which
// must hold zero; conf gets n*dim, hang n*2dim and hcon 4 x that entries at most.
// pub (nullable; host memory mapped for the device): the block that finishes last (counted in
// *done, which must hold zero) copies words[0..nwords) there, then writes seq to pub[nwords], so
// the host can read the adaptation's counts without a copy and a stream synchronisation.
struct FaceLists {
  int32_t* conf = nullptr;
  int32_t* hang = nullptr;
  int32_t* hcon = nullptr;
  unsigned long long* count = nullptr;
  int64_t* pub = nullptr;
  const int64_t* words = nullptr;
  int nwords = 0;
  int64_t seq = 0;
  unsigned long long* done = nullptr;
  KeyIndex index;  // of the keys (nullable): the searches use it
};
int tree_conn(int dim, const KG& g, const uint64_t* d_keys, int64_t n, const int64_t* d_n, int32_t* d_nbr,
              int8_t* d_ftype, int8_t* d_slot, int32_t* d_contrib, int32_t* d_bad, cudaStream_t s,
              Err* err, int64_t* d_fcnt = nullptr, const FaceLists& L = FaceLists{});
// sets *d_bad (not cleared here) unless keys are a complete sorted linear tree with depths in [Dlo, Dhi]
int tree_validate_async(int dim, const KG& g, const uint64_t* d_keys, int64_t n, int Dlo, int Dhi,
                        int32_t* d_bad, cudaStream_t s, Err* err);
// checks that keys are a complete sorted linear tree with depths in [Dlo, Dhi]
int tree_validate(int dim, const KG& g, const uint64_t* d_keys, int64_t n, int Dlo, int Dhi,
                  bool* ok, Alloc& A, cudaStream_t s, Err* err);

// ---------------------------------------------------------------------------------------------
// FR operators (host-built, passed to kernels by value)
// ---------------------------------------------------------------------------------------------
constexpr int NPMAX = 5;
struct DevOps {
  double x[NPMAX], w[NPMAX];
  double D[NPMAX][NPMAX];    // D[i][j] = l_j'(x_i)
  double Dt[NPMAX][NPMAX];   // D folded with the correction: D - gL lm^T - gR lp^T
  double lm[NPMAX], lp[NPMAX];
  double gL[NPMAX], gR[NPMAX];
  double I[2][NPMAX][NPMAX]; // I[h][i][j] = l_j((x_i + 2h - 1)/2): parent -> half h
  double P[2][NPMAX][NPMAX]; // P[h][j][i] = (1/2)(w_i/w_j) I[h][i][j]: half h -> parent (L2)
};
int build_ops(int p, DevOps* o);

struct DevProblem {
  double L, gamma, rho_inf, p_inf, uinf[3];
  int nvort;
  double vort[16][4];
};

}  // namespace frg
