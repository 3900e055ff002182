// fr_prim.cu -- device-wide primitives without CUB: exclusive scan (reduce-then-scan, no
// inter-block waits), stable LSD radix sort of uint64 keys (warp-match ranking), device memory.
#include <atomic>
#include <cstdio>

#include "fr_internal.cuh"

namespace frg {

// ---------------------------------------------------------------------------------------------
// errors and allocation
// ---------------------------------------------------------------------------------------------
int set_error(Err* e, int code, const std::string& msg) {
  if (e) {
    e->code = code;
    e->msg = msg;
  }
  return code;
}

int64_t& launch_counter() {
  static int64_t n = 0;
  return n;
}

Err* global_err() {
  static thread_local Err e;
  return &e;
}

static void* raw_get(const fr_allocator* user, cudaStream_t stream, size_t bytes) {
  void* p = nullptr;
  if (user && user->alloc) {
    p = user->alloc(bytes, (void*)stream, user->ctx);
  } else if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  return p;
}

static void raw_put(const fr_allocator* user, cudaStream_t stream, void* p) {
  if (user && user->free)
    user->free(p, (void*)stream, user->ctx);
  else
    cudaFreeAsync(p, stream);
}

void* Alloc::get(size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) / 256 * 256;
  if (bytes > 65536) {
    // eight size classes per power of two (at most 12.5% slack): a request that grows by a few
    // leaves from one adaptation to the next then finds last time's block in the cache
    int lg = 63 - __builtin_clzll(bytes);
    size_t step = size_t(1) << (lg - 3);
    bytes = (bytes + step - 1) / step * step;
  }
  if (cache) {
    // smallest cached block that fits without wasting more than half of it
    size_t best = size_t(-1);
    for (size_t k = 0; k < cache->free_blocks.size(); ++k) {
      size_t sz = cache->free_blocks[k].second;
      if (sz >= bytes && sz <= 2 * bytes + 4096 && (best == size_t(-1) || sz < cache->free_blocks[best].second))
        best = k;
    }
    if (best != size_t(-1)) {
      auto blk = cache->free_blocks[best];
      cache->free_blocks.erase(cache->free_blocks.begin() + long(best));
      cache->live.push_back(blk);
      return blk.first;
    }
  }
  void* p = raw_get(user, stream, bytes);
  if (p && cache) cache->live.push_back({p, bytes});
  return p;
}

void Alloc::put(void* p) {
  if (!p) return;
  if (cache) {
    for (size_t k = 0; k < cache->live.size(); ++k)
      if (cache->live[k].first == p) {
        cache->free_blocks.push_back(cache->live[k]);
        cache->live.erase(cache->live.begin() + long(k));
        return;
      }
  }
  raw_put(user, stream, p);
}

void Alloc::release_cache() {
  if (!cache) return;
  for (auto& b : cache->free_blocks) raw_put(user, stream, b.first);
  cache->free_blocks.clear();
}

int read_i64(const int64_t* d, int64_t* h, cudaStream_t s, Err* err) {
  FR_CUDA(err, cudaMemcpyAsync(h, d, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  FR_CUDA(err, cudaStreamSynchronize(s));
  return 0;
}

// ---------------------------------------------------------------------------------------------
// exclusive scan: each block scans a tile of SCAN_T*SCAN_I items held blocked in registers,
// block totals are scanned recursively, then added back.
// ---------------------------------------------------------------------------------------------
constexpr int SCAN_T = 256, SCAN_I = 8, SCAN_TILE = SCAN_T * SCAN_I;

template <class TIn>
__global__ void __launch_bounds__(SCAN_T) k_scan_tile(const TIn* __restrict__ in,
                                                      int64_t* __restrict__ out, int64_t n,
                                                      int64_t* __restrict__ sums) {
  pdl_wait_then_release();
  __shared__ int64_t s_warp[SCAN_T / 32];
  __shared__ TIn s_in[SCAN_TILE];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int64_t base = int64_t(blockIdx.x) * SCAN_TILE;
  for (int k = t; k < SCAN_TILE; k += SCAN_T) {  // coalesced load, then blocked use
    int64_t idx = base + k;
    s_in[k] = idx < n ? in[idx] : TIn(0);
  }
  __syncthreads();
  int64_t v[SCAN_I], run = 0;
#pragma unroll
  for (int k = 0; k < SCAN_I; ++k) {
    v[k] = run;
    run += int64_t(s_in[t * SCAN_I + k]);
  }
  int64_t incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int64_t w = lane < SCAN_T / 32 ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < SCAN_T / 32) s_warp[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  int64_t excl_thread = incl - run + (wid ? s_warp[wid - 1] : 0);
  __syncthreads();
  int64_t* s_out = reinterpret_cast<int64_t*>(s_in);  // reuse only if TIn is 8 bytes
  if (sizeof(TIn) == 8) {
#pragma unroll
    for (int k = 0; k < SCAN_I; ++k) s_out[t * SCAN_I + k] = v[k] + excl_thread;
    __syncthreads();
    for (int k = t; k < SCAN_TILE; k += SCAN_T) {
      int64_t idx = base + k;
      if (idx < n) out[idx] = s_out[k];
    }
  } else {
#pragma unroll
    for (int k = 0; k < SCAN_I; ++k) {
      int64_t idx = base + t * SCAN_I + k;
      if (idx < n) out[idx] = v[k] + excl_thread;
    }
  }
  if (t == SCAN_T - 1) sums[blockIdx.x] = excl_thread + run;
}

__global__ void k_scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ offs) {
  pdl_wait_then_release();
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] += offs[i / SCAN_TILE];
}

// second pass for up to SCAN_PREFIX_MAX tiles: every 256-element block lies inside one tile and
// sums the totals of the tiles before it itself (no third launch); block 0 also writes the total
constexpr int64_t SCAN_PREFIX_MAX = 256;
__global__ void __launch_bounds__(256) k_scan_add_prefix(int64_t* __restrict__ out, int64_t n,
                                                         const int64_t* __restrict__ sums, int64_t nb,
                                                         int64_t* __restrict__ total) {
  pdl_wait_then_release();
  __shared__ int64_t red[256];
  const int t = threadIdx.x;
  const int64_t i0 = int64_t(blockIdx.x) * 256;
  const int64_t tile = i0 / SCAN_TILE;
  int64_t a = 0;
  for (int64_t k = t; k < tile; k += 256) a += sums[k];
  red[t] = a;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (t < st) red[t] += red[t + st];
    __syncthreads();
  }
  const int64_t prefix = red[0];
  if (i0 + t < n) out[i0 + t] += prefix;
  if (blockIdx.x == 0) {
    __syncthreads();
    a = 0;
    for (int64_t k = t; k < nb; k += 256) a += sums[k];
    red[t] = a;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
      if (t < st) red[t] += red[t + st];
      __syncthreads();
    }
    if (t == 0) *total = red[0];
  }
}

template <class TIn>
static int scan_impl(const TIn* d_in, int64_t* d_out, int64_t n, int64_t* d_total, Scratch& S,
                     cudaStream_t s, Err* err) {
  if (n <= 0) {
    FR_CUDA(err, cudaMemsetAsync(d_total, 0, sizeof(int64_t), s));
    return 0;
  }
  int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nb == 1) {
    launch_dependent(k_scan_tile<TIn>, 1, SCAN_T, s, d_in, d_out, n, d_total);
    FR_LAUNCH_CHECK(err);
    return 0;
  }
  if (nb <= SCAN_PREFIX_MAX) {
    int64_t* sums1 = S.get<int64_t>(nb);
    if (!sums1) return set_error(err, FR_ENOMEM, "scan scratch");
    launch_dependent(k_scan_tile<TIn>, unsigned(nb), SCAN_T, s, d_in, d_out, n, sums1);
    FR_LAUNCH_CHECK(err);
    launch_dependent(k_scan_add_prefix, unsigned((n + 255) / 256), 256, s, d_out, n,
                     static_cast<const int64_t*>(sums1), nb, d_total);
    FR_LAUNCH_CHECK(err);
    return 0;
  }
  int64_t* sums = S.get<int64_t>(nb);
  int64_t* offs = S.get<int64_t>(nb);
  if (!sums || !offs) return set_error(err, FR_ENOMEM, "scan scratch");
  k_scan_tile<TIn><<<unsigned(nb), SCAN_T, 0, s>>>(d_in, d_out, n, sums);
  FR_LAUNCH_CHECK(err);
  FR_TRY(scan_impl<int64_t>(sums, offs, nb, d_total, S, s, err));
  k_scan_add<<<unsigned((n + 255) / 256), 256, 0, s>>>(d_out, n, offs);
  FR_LAUNCH_CHECK(err);
  return 0;
}

template <class TIn>
static int scan_local_impl(const TIn* d_in, int64_t* d_out, int64_t n, int64_t* d_total, Scratch& S,
                           cudaStream_t s, Err* err, Offs* O) {
  static_assert(SCAN_TILE == SCAN_TILE_ITEMS, "tile size");
  const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (n <= 0 || nb == 1 || nb > SCAN_PREFIX_MAX) {
    *O = Offs{d_out, nullptr, 0, d_total};
    return scan_impl<TIn>(d_in, d_out, n, d_total, S, s, err);
  }
  int64_t* sums = S.get<int64_t>(nb);
  if (!sums) return set_error(err, FR_ENOMEM, "scan scratch");
  launch_dependent(k_scan_tile<TIn>, unsigned(nb), SCAN_T, s, d_in, d_out, n, sums);
  FR_LAUNCH_CHECK(err);
  *O = Offs{d_out, sums, nb, d_total};
  return 0;
}
int scan_counts_local(const int32_t* d_in, int64_t* d_out, int64_t n, int64_t* d_total, Scratch& S,
                      cudaStream_t s, Err* err, Offs* O) {
  return scan_local_impl<int32_t>(d_in, d_out, n, d_total, S, s, err, O);
}
int scan_counts64_local(const int64_t* d_in, int64_t* d_out, int64_t n, int64_t* d_total, Scratch& S,
                        cudaStream_t s, Err* err, Offs* O) {
  return scan_local_impl<int64_t>(d_in, d_out, n, d_total, S, s, err, O);
}

int scan_counts(const int32_t* d_in, int64_t* d_out, int64_t n, int64_t* d_total, Scratch& S,
                cudaStream_t s, Err* err) {
  return scan_impl<int32_t>(d_in, d_out, n, d_total, S, s, err);
}

int scan_counts64(const int64_t* d_in, int64_t* d_out, int64_t n, int64_t* d_total, Scratch& S,
                  cudaStream_t s, Err* err) {
  return scan_impl<int64_t>(d_in, d_out, n, d_total, S, s, err);
}

// ---------------------------------------------------------------------------------------------
// LSD radix sort, 8-bit digits.  Pass = per-tile digit histogram -> exclusive scan of the
// digit-major histogram -> stable scatter.  Inside a tile each warp ranks its contiguous chunk
// round by round with __match_any_sync; per-warp digit counts give the cross-warp offsets.
// ---------------------------------------------------------------------------------------------
constexpr int RS_WARPS = 8, RS_T = RS_WARPS * 32, RS_ITEMS = 8;
constexpr int RS_CHUNK = 32 * RS_ITEMS, RS_TILE = RS_WARPS * RS_CHUNK;

__global__ void __launch_bounds__(RS_T) k_rs_hist(const uint64_t* __restrict__ keys, int64_t n,
                                                  int shift, int32_t* __restrict__ hist, int nb) {
  __shared__ int32_t h[256];
  const int t = threadIdx.x;
  h[t] = 0;
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * RS_TILE;
  for (int k = t; k < RS_TILE; k += RS_T) {
    int64_t idx = base + k;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1);
  }
  __syncthreads();
  hist[int64_t(t) * nb + blockIdx.x] = h[t];
}

__global__ void __launch_bounds__(RS_T) k_rs_scatter(const uint64_t* __restrict__ in,
                                                     uint64_t* __restrict__ out, int64_t n,
                                                     int shift, const int64_t* __restrict__ offs,
                                                     int nb) {
  __shared__ int32_t wcnt[RS_WARPS][256];
  __shared__ int64_t gofs[256];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (int k = t; k < RS_WARPS * 256; k += RS_T) (&wcnt[0][0])[k] = 0;
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  const int64_t base = int64_t(blockIdx.x) * RS_TILE + int64_t(w) * RS_CHUNK;
  uint64_t key[RS_ITEMS];
  int dig[RS_ITEMS], rank[RS_ITEMS];
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    int64_t idx = base + r * 32 + lane;
    bool valid = idx < n;
    key[r] = valid ? in[idx] : 0ull;
    dig[r] = valid ? int((key[r] >> shift) & 255u) : 256;
    unsigned peers = __match_any_sync(0xffffffffu, dig[r]);
    int before = valid ? wcnt[w][dig[r]] : 0;
    rank[r] = before + __popc(peers & lt);
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) wcnt[w][dig[r]] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {
    int d = t;  // RS_T == 256: one digit per thread
    int32_t run = 0;
    for (int ww = 0; ww < RS_WARPS; ++ww) {
      int32_t c = wcnt[ww][d];
      wcnt[ww][d] = run;
      run += c;
    }
    gofs[d] = offs[int64_t(d) * nb + blockIdx.x];
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    if (dig[r] < 256) out[gofs[dig[r]] + wcnt[w][dig[r]] + rank[r]] = key[r];
  }
}

int radix_sort_keys(uint64_t* d_keys, uint64_t* d_tmp, int64_t n, int bits, Scratch& S,
                    cudaStream_t s, Err* err) {
  if (n <= 1) return 0;
  int64_t nb64 = (n + RS_TILE - 1) / RS_TILE;
  if (nb64 > (int64_t(1) << 22)) return set_error(err, FR_EINVAL, "radix sort: too many keys");
  int nb = int(nb64);
  int32_t* hist = S.get<int32_t>(size_t(256) * nb);
  int64_t* offs = S.get<int64_t>(size_t(256) * nb);
  int64_t* total = S.get<int64_t>(1);
  if (!hist || !offs || !total) return set_error(err, FR_ENOMEM, "radix sort scratch");
  uint64_t* src = d_keys;
  uint64_t* dst = d_tmp;
  int passes = (bits + 7) / 8;
  for (int ps = 0; ps < passes; ++ps) {
    int shift = ps * 8;
    k_rs_hist<<<nb, RS_T, 0, s>>>(src, n, shift, hist, nb);
    FR_LAUNCH_CHECK(err);
    FR_TRY(scan_counts(hist, offs, int64_t(256) * nb, total, S, s, err));
    k_rs_scatter<<<nb, RS_T, 0, s>>>(src, dst, n, shift, offs, nb);
    FR_LAUNCH_CHECK(err);
    uint64_t* tmp = src;
    src = dst;
    dst = tmp;
  }
  if (src != d_keys)
    FR_CUDA(err, cudaMemcpyAsync(d_keys, src, size_t(n) * 8, cudaMemcpyDeviceToDevice, s));
  return 0;
}


// ---------------------------------------------------------------------------------------------
// Allocation-free variant of the key sort (fr_keys_sort_noalloc).  Its scratch is one file-scope
// device array, sized for FR_NOALLOC_SORT_MAX_KEYS keys and resident on every device that loads
// the library until the process exits.  In host code the array's name is only a host-side handle,
// so its device address is looked up once per device with cudaGetSymbolAddress.
// ---------------------------------------------------------------------------------------------
namespace {

constexpr int64_t NA_MAX = FR_NOALLOC_SORT_MAX_KEYS;
constexpr int64_t NA_NB = (NA_MAX + RS_TILE - 1) / RS_TILE;            // radix tiles
constexpr int64_t NA_HIST = 256 * NA_NB;                               // digit counters
constexpr int64_t NA_SNB = (NA_HIST + SCAN_TILE - 1) / SCAN_TILE;      // scan tiles (<= SCAN_TILE)
static_assert(NA_SNB <= SCAN_TILE, "two-level scan must cover the histogram");
constexpr size_t na_align(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t NA_OFF_TMP = 0;
constexpr size_t NA_OFF_HIST = NA_OFF_TMP + na_align(sizeof(uint64_t) * NA_MAX);
constexpr size_t NA_OFF_OFFS = NA_OFF_HIST + na_align(sizeof(int32_t) * NA_HIST);
constexpr size_t NA_OFF_SUMS = NA_OFF_OFFS + na_align(sizeof(int64_t) * NA_HIST);
constexpr size_t NA_OFF_SOFF = NA_OFF_SUMS + na_align(sizeof(int64_t) * NA_SNB);
constexpr size_t NA_OFF_TOT = NA_OFF_SOFF + na_align(sizeof(int64_t) * NA_SNB);
constexpr size_t NA_BYTES = NA_OFF_TOT + 256;

static __device__ __align__(256) unsigned char g_noalloc_sort_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 64;
// per device, the looked-up address; atomic, because host threads may make their first calls on
// a device at the same time (each looks the address up and stores the same value)
std::atomic<unsigned char*> g_noalloc_ptr[NA_MAX_DEVICES];

// device address of the scratch array on the current device (looked up on first use)
int noalloc_scratch(unsigned char** out, Err* err) {
  int dev = 0;
  FR_CUDA(err, cudaGetDevice(&dev));
  if (dev < 0 || dev >= NA_MAX_DEVICES) return set_error(err, FR_EINVAL, "device index too large");
  unsigned char* p = g_noalloc_ptr[dev].load(std::memory_order_acquire);
  if (!p) {
    void* q = nullptr;
    cudaError_t ce = cudaGetSymbolAddress(&q, g_noalloc_sort_scratch);
    if (ce != cudaSuccess || !q)
      return set_error(err, FR_ECUDA, std::string("cudaGetSymbolAddress(sort scratch): ") +
                                          cudaGetErrorString(ce));
    p = static_cast<unsigned char*>(q);
    g_noalloc_ptr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return 0;
}

}  // namespace

int radix_sort_keys_noalloc(uint64_t* d_keys, int64_t n, int bits, cudaStream_t s, Err* err) {
  if (n < 0) return set_error(err, FR_EINVAL, "n < 0");
  if (n > NA_MAX)
    return set_error(err, FR_EINVAL, "fr_keys_sort_noalloc: n exceeds FR_NOALLOC_SORT_MAX_KEYS");
  if (n <= 1) return 0;
  unsigned char* base = nullptr;
  FR_TRY(noalloc_scratch(&base, err));
  uint64_t* tmp = reinterpret_cast<uint64_t*>(base + NA_OFF_TMP);
  int32_t* hist = reinterpret_cast<int32_t*>(base + NA_OFF_HIST);
  int64_t* offs = reinterpret_cast<int64_t*>(base + NA_OFF_OFFS);
  int64_t* sums = reinterpret_cast<int64_t*>(base + NA_OFF_SUMS);
  int64_t* soff = reinterpret_cast<int64_t*>(base + NA_OFF_SOFF);
  int64_t* tot = reinterpret_cast<int64_t*>(base + NA_OFF_TOT);
  // every scratch word read below is written earlier in the same call (histograms by k_rs_hist,
  // offsets by the scan), so nothing has to be cleared between calls
  int nb = int((n + RS_TILE - 1) / RS_TILE);
  int64_t nh = int64_t(256) * nb;
  int64_t snb = (nh + SCAN_TILE - 1) / SCAN_TILE;
  uint64_t* src = d_keys;
  uint64_t* dst = tmp;
  for (int ps = 0; ps < (bits + 7) / 8; ++ps) {
    int shift = ps * 8;
    k_rs_hist<<<nb, RS_T, 0, s>>>(src, n, shift, hist, nb);
    FR_LAUNCH_CHECK(err);
    if (snb == 1) {
      k_scan_tile<int32_t><<<1, SCAN_T, 0, s>>>(hist, offs, nh, tot);
      FR_LAUNCH_CHECK(err);
    } else {
      k_scan_tile<int32_t><<<unsigned(snb), SCAN_T, 0, s>>>(hist, offs, nh, sums);
      FR_LAUNCH_CHECK(err);
      k_scan_tile<int64_t><<<1, SCAN_T, 0, s>>>(sums, soff, snb, tot);
      FR_LAUNCH_CHECK(err);
      k_scan_add<<<unsigned((nh + 255) / 256), 256, 0, s>>>(offs, nh, soff);
      FR_LAUNCH_CHECK(err);
    }
    k_rs_scatter<<<nb, RS_T, 0, s>>>(src, dst, n, shift, offs, nb);
    FR_LAUNCH_CHECK(err);
    uint64_t* t2 = src;
    src = dst;
    dst = t2;
  }
  if (src != d_keys)
    FR_CUDA(err, cudaMemcpyAsync(d_keys, src, size_t(n) * 8, cudaMemcpyDeviceToDevice, s));
  return 0;
}

}  // namespace frg

extern "C" int fr_keys_sort_noalloc(int dim, int Dmax, uint64_t* d_keys, int64_t n, void* stream) {
  frg::Err* err = frg::global_err();
  if ((dim != 2 && dim != 3) || Dmax < 1 || Dmax > 30)
    return frg::set_error(err, FR_EINVAL, "dim/Dmax out of range");
  int bits = dim * Dmax + frg::depth_bits(Dmax);
  if (bits > 63) return frg::set_error(err, FR_EINVAL, "dim*Dmax + depth bits exceeds 63");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  FR_TRY(frg::radix_sort_keys_noalloc(d_keys, n, bits, s, err));
  FR_CUDA(err, cudaStreamSynchronize(s));
  return 0;
}

