// Runtime pieces of the library: status strings, error messages, launch
// counter, the stream-ordered memory pool and a device-wide exclusive scan.
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "ph_internal.cuh"

namespace ph {

std::atomic<int64_t> g_launches{0};

static thread_local char t_msg[256] = "";

void set_error_message(const char* what, cudaError_t e) {
  snprintf(t_msg, sizeof t_msg, "%s: %s", what, cudaGetErrorString(e));
}

void set_error_text(const char* text) { snprintf(t_msg, sizeof t_msg, "%s", text); }

ph_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PH_OK;
  set_error_message(what, e);
  return e == cudaErrorMemoryAllocation ? PH_ERR_NOMEM : PH_ERR_CUDA;
}

// One pool per device, created on first use.  Its release threshold is the
// maximum, so memory freed in stream order is reused by later allocations
// instead of being returned to the driver at every synchronisation.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[64];
static bool g_pool_ok[64];

static cudaError_t pool_for(int dev, cudaMemPool_t* out) {
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool_ok[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaError_t e = cudaMemPoolCreate(&g_pools[dev], &props);
    if (e != cudaSuccess) return e;
    uint64_t thr = ~0ull;
    e = cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &thr);
    if (e != cudaSuccess) return e;
    // A block freed on another stream is reused only once its free has
    // completed, never by making this stream wait for that one: calls on
    // different streams (several host threads) must not serialise through
    // the pool.  The pool grows instead.
    int no = 0;
    e = cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolReuseAllowInternalDependencies, &no);
    if (e != cudaSuccess) return e;
    g_pool_ok[dev] = true;
  }
  *out = g_pools[dev];
  return cudaSuccess;
}

// Test hook (ph_test_fail_alloc): the number of pool allocations still to
// succeed before one fails; negative = never fail.
static std::atomic<int64_t> g_fail_alloc_after{-1};

cudaError_t alloc_bytes(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (g_fail_alloc_after.load(std::memory_order_relaxed) >= 0 && g_fail_alloc_after.fetch_sub(1) == 0)
    return cudaErrorMemoryAllocation;  // the injected failure (once)
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaMemPool_t pool;
  e = pool_for(dev, &pool);
  if (e != cudaSuccess) return e;
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

void free_async(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

// ---------------------------------------------------------------------------
// Exclusive scan: reduce tiles -> scan tile sums (one block) -> scan tiles.
// ---------------------------------------------------------------------------
constexpr int SCAN_T = 256;
constexpr int SCAN_I = 16;  // a multiple of 4 (16-byte accesses)
constexpr int SCAN_TILE = SCAN_T * SCAN_I;

template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Exclusive scan of one value per thread across the block; returns the
// exclusive prefix and writes the block total to *total.
template <class T, int NT>
__device__ __forceinline__ T block_excl_scan(T v, T* total) {
  __shared__ T warp_sums[NT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T inc = warp_incl_scan(v);
  if (lane == 31) warp_sums[w] = inc;
  __syncthreads();
  if (w == 0) {
    T x = (lane < NT / 32) ? warp_sums[lane] : T(0);
    x = warp_incl_scan(x);
    if (lane < NT / 32) warp_sums[lane] = x;
  }
  __syncthreads();
  T before = (w > 0 ? warp_sums[w - 1] : T(0)) + inc - v;
  *total = warp_sums[NT / 32 - 1];
  __syncthreads();
  return before;
}

// Single-pass exclusive scan with decoupled look-back (Merrill and Garland,
// "Single-pass Parallel Prefix Scan with Decoupled Look-back", 2016).  Tiles
// of SCAN_TILE elements take ids from an atomic counter in the order the
// blocks start, so every predecessor of a tile is running or done.  A tile
// publishes its aggregate (flag 1); its first warp then reads the state of
// 32 predecessors at a time, adds the values up to the nearest one that
// carries an inclusive prefix (flag 2), and the tile publishes its own
// inclusive prefix.  State word: flag in bits 62..63, value in bits 0..61
// (inputs are non-negative counts).
constexpr unsigned long long kScanAgg = 1ull << 62, kScanInc = 2ull << 62, kScanVal = (1ull << 62) - 1;
constexpr int kScanSpinLimit = 1 << 20;  // unready polls before giving up (>= 32 ns apart)
// Test hook (ph_test_scan_withhold): scans run with tile 1 never publishing
// its state and this short poll limit, so that a look-back wait runs out.
constexpr int kScanTestSpinLimit = 1 << 12;
static std::atomic<int> g_scan_withhold{0};

__global__ void __launch_bounds__(SCAN_T) k_scan(const int32_t* in, int32_t* out, int64_t nmax,
                                                  const int64_t* __restrict__ d_len, int64_t len_add,
                                                  int64_t* __restrict__ d_total, unsigned long long* state,
                                                  unsigned* counter, unsigned* status,
                                                  const int4* __restrict__ mates, int64_t nmates,
                                                  int spin_limit, int64_t withhold) {
  __shared__ unsigned s_tile;
  __shared__ int64_t s_prefix;
  if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1u);
  __syncthreads();
  const int64_t n = d_len ? min(nmax, *d_len + len_add) : nmax;
  const int64_t tile = s_tile;
  const int64_t last = n > 0 ? (n - 1) / SCAN_TILE : 0;
  if (tile > last) return;  // past the device-side length: nobody looks back at it
  const int64_t base = tile * SCAN_TILE + (int64_t)threadIdx.x * SCAN_I;
  const bool vec = base + SCAN_I <= n && ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
  int32_t v[SCAN_I];
  if (mates) {
    // first occurrences per tet, from the face mates: the block loads the
    // tile's mates with consecutive threads on consecutive tets (coalesced),
    // counts them, and hands each thread its SCAN_I consecutive counts through
    // shared memory (one pad word per 32, so both passes are free of bank
    // conflicts)
    __shared__ int32_t s_cnt[SCAN_TILE + SCAN_TILE / 32];
#pragma unroll
    for (int q = 0; q < SCAN_I; ++q) {
      const int j = q * SCAN_T + threadIdx.x;
      const int64_t t = tile * SCAN_TILE + j;
      s_cnt[j + (j >> 5)] = t < nmates && t < n ? first_occurrences(mates[t], (int)(4 * t)) : 0;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < SCAN_I; ++i) {
      const int j = threadIdx.x * SCAN_I + i;
      v[i] = s_cnt[j + (j >> 5)];
    }
  } else if (vec) {
#pragma unroll
    for (int q = 0; q < SCAN_I / 4; ++q) {
      const int4 a = *reinterpret_cast<const int4*>(in + base + 4 * q);
      v[4 * q] = a.x;
      v[4 * q + 1] = a.y;
      v[4 * q + 2] = a.z;
      v[4 * q + 3] = a.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < SCAN_I; ++i) v[i] = base + i < n ? in[base + i] : 0;
  }
  int64_t sum = 0;
#pragma unroll
  for (int i = 0; i < SCAN_I; ++i) sum += v[i];
  int64_t tot;
  const int64_t ex = block_excl_scan<int64_t, SCAN_T>(sum, &tot);
  if (threadIdx.x < 32) {
    volatile unsigned long long* st = state;
    const int lane = threadIdx.x;
    int64_t prefix = 0;
    const bool publish = tile != withhold;
    if (tile > 0) {
      if (lane == 0 && publish) st[tile] = kScanAgg | (unsigned long long)tot;
      int spins = 0;
      for (int64_t p = tile - 1; p >= 0;) {
        const int64_t q = p - lane;  // lane 0 is the nearest predecessor
        unsigned long long w = kScanInc;  // before tile 0: an inclusive prefix of 0
        if (q >= 0) w = st[q];
        while (__any_sync(0xFFFFFFFFu, (w >> 62) == 0)) {
          if (++spins > spin_limit) break;
          __nanosleep(32);
          if ((w >> 62) == 0) w = st[q];
        }
        if (spins > spin_limit) {  // a predecessor never published: give up, flagged
          if (lane == 0 && status) ph_flag(status, PH_ERR_TIMEOUT);
          break;
        }
        const unsigned inc = __ballot_sync(0xFFFFFFFFu, (w >> 62) == 2);
        const int stop = inc ? __ffs(inc) - 1 : 31;  // add lanes 0..stop
        int64_t x = lane <= stop ? (int64_t)(w & kScanVal) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
        prefix += __shfl_sync(0xFFFFFFFFu, x, 0);
        if (inc) break;
        p -= 32;
      }
    }
    if (lane == 0) {
      __threadfence();
      if (publish) st[tile] = kScanInc | (unsigned long long)(prefix + tot);
      s_prefix = prefix;
      if (tile == last && d_total) *d_total = prefix + tot;
    }
  }
  __syncthreads();
  int64_t run = s_prefix + ex;
  int32_t o[SCAN_I];
#pragma unroll
  for (int i = 0; i < SCAN_I; ++i) {
    o[i] = (int32_t)run;
    run += v[i];
  }
  if (vec) {
#pragma unroll
    for (int q = 0; q < SCAN_I / 4; ++q)
      *reinterpret_cast<int4*>(out + base + 4 * q) = make_int4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
  } else {
#pragma unroll
    for (int i = 0; i < SCAN_I; ++i)
      if (base + i < n) out[base + i] = o[i];
  }
}

size_t scan_state_words(int64_t n) {
  const int64_t ntiles = n > 0 ? (n + SCAN_TILE - 1) / SCAN_TILE : 1;
  return (size_t)ntiles + 1;  // tile states, then the tile counter
}

ph_status exclusive_scan(const int32_t* in, int32_t* out, int64_t n, int64_t* d_total, cudaStream_t s,
                         unsigned* status, const int64_t* d_len, int64_t len_add, unsigned long long* given,
                         const int4* mates, int64_t nmates) {
  int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (ntiles < 1) ntiles = 1;
  unsigned long long* state = given;  // ntiles words, then the tile counter
  cudaError_t e = cudaSuccess;
  if (!state) {
    e = alloc(&state, (size_t)ntiles + 1, s);
    if (e != cudaSuccess) return cuda_status(e, "scan alloc");
    e = cudaMemsetAsync(state, 0, sizeof(unsigned long long) * (ntiles + 1), s);
  }
  if (e == cudaSuccess) {
    KernelTimer kt("k_scan", s, 2);
    const bool withhold = g_scan_withhold.load(std::memory_order_relaxed) != 0;
    k_scan<<<(unsigned)ntiles, SCAN_T, 0, s>>>(in, out, n, d_len, len_add, d_total, state,
                                               reinterpret_cast<unsigned*>(state + ntiles), status, mates,
                                               nmates, withhold ? kScanTestSpinLimit : kScanSpinLimit,
                                               withhold ? 1 : -1);
    e = launched();
    kt.stop();
  }
  if (!given) free_async(state, s);
  return cuda_status(e, "scan");
}

}  // namespace ph

extern "C" const char* ph_status_string(ph_status s) {
  switch (s) {
    case PH_OK: return "PH_OK";
    case PH_ERR_ARG: return "PH_ERR_ARG";
    case PH_ERR_DEGENERATE: return "PH_ERR_DEGENERATE";
    case PH_ERR_NONMANIFOLD: return "PH_ERR_NONMANIFOLD";
    case PH_ERR_OVERFLOW: return "PH_ERR_OVERFLOW";
    case PH_ERR_NOMEM: return "PH_ERR_NOMEM";
    case PH_ERR_CUDA: return "PH_ERR_CUDA";
    case PH_ERR_NOT_CONVERGED: return "PH_ERR_NOT_CONVERGED";
    case PH_ERR_TIMEOUT: return "PH_ERR_TIMEOUT";
  }
  return "PH_ERR_UNKNOWN";
}

extern "C" const char* ph_last_error_message(void) { return ph::t_msg; }

extern "C" int64_t ph_launch_count(void) { return ph::g_launches.load(); }

// --- kernel timing ---------------------------------------------------------
namespace ph {
namespace {
struct TimedLaunch {
  const char* name;
  cudaEvent_t a, b;
};
std::atomic<unsigned> g_timing{0};  // mask of timed categories
std::mutex g_timing_mu;
std::vector<TimedLaunch> g_timed;                          // recorded, not yet read
std::map<std::string, std::pair<double, int64_t>> g_time;  // name -> (ms, launches)
std::vector<cudaEvent_t> g_event_pool;                     // created once, reused (device of first use)

cudaEvent_t take_event() {
  {
    std::lock_guard<std::mutex> lk(g_timing_mu);
    if (!g_event_pool.empty()) {
      cudaEvent_t e = g_event_pool.back();
      g_event_pool.pop_back();
      return e;
    }
  }
  cudaEvent_t e = nullptr;
  return cudaEventCreate(&e) == cudaSuccess ? e : nullptr;
}

void give_event(cudaEvent_t e) {  // caller holds g_timing_mu
  if (e) g_event_pool.push_back(e);
}
}  // namespace

KernelTimer::KernelTimer(const char* name, cudaStream_t s, unsigned category) : name_(name), s_(s) {
  if (!(g_timing.load(std::memory_order_relaxed) & category)) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  a_ = take_event();
  b_ = take_event();
  if (!a_ || !b_ || cudaEventRecord(a_, s) != cudaSuccess) {
    std::lock_guard<std::mutex> lk(g_timing_mu);
    give_event(a_);
    give_event(b_);
    a_ = b_ = nullptr;
  }
}

void KernelTimer::stop() {
  if (!a_) return;
  const bool ok = cudaEventRecord(b_, s_) == cudaSuccess;
  std::lock_guard<std::mutex> lk(g_timing_mu);
  if (ok) {
    g_timed.push_back({name_, a_, b_});
  } else {
    give_event(a_);
    give_event(b_);
  }
  a_ = b_ = nullptr;
}
}  // namespace ph

extern "C" ph_status ph_timing_enable(int on) {
  if (on) {  // stock the event pool now, so that timing does not create events between launches
    constexpr size_t kStock = 4096;
    std::vector<cudaEvent_t> fresh;
    {
      std::lock_guard<std::mutex> lk(ph::g_timing_mu);
      const size_t have = ph::g_event_pool.size() + 2 * ph::g_timed.size();
      if (have < kStock) fresh.resize(kStock - have, nullptr);
    }
    for (cudaEvent_t& e : fresh)
      if (cudaEventCreate(&e) != cudaSuccess) return ph::cuda_status(cudaErrorMemoryAllocation, "ph_timing_enable");
    std::lock_guard<std::mutex> lk(ph::g_timing_mu);
    for (cudaEvent_t e : fresh) ph::g_event_pool.push_back(e);
  }
  ph::g_timing.store(on < 0 ? 0u : (unsigned)on);
  return PH_OK;
}

extern "C" ph_status ph_kernel_time(const char* kernel, int reset, double* ms, int64_t* launches) {
  if (!kernel) return PH_ERR_ARG;
  std::lock_guard<std::mutex> lk(ph::g_timing_mu);
  cudaError_t err = cudaSuccess;
  std::vector<ph::TimedLaunch> keep;
  for (const ph::TimedLaunch& t : ph::g_timed) {
    if (strcmp(t.name, kernel) != 0) {
      keep.push_back(t);
      continue;
    }
    float f = 0.f;
    cudaError_t e = cudaEventSynchronize(t.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&f, t.a, t.b);
    if (e == cudaSuccess) {
      auto& acc = ph::g_time[kernel];
      acc.first += f;
      acc.second += 1;
    } else if (err == cudaSuccess) {
      err = e;
    }
    ph::give_event(t.a);
    ph::give_event(t.b);
  }
  ph::g_timed.swap(keep);
  auto it = ph::g_time.find(kernel);
  if (ms) *ms = it == ph::g_time.end() ? 0.0 : it->second.first;
  if (launches) *launches = it == ph::g_time.end() ? 0 : it->second.second;
  if (reset && it != ph::g_time.end()) ph::g_time.erase(it);
  return ph::cuda_status(err, "ph_kernel_time");
}

namespace {
__global__ void k_rcp(const double* __restrict__ x, int64_t n, double* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = ph::rcp_newton(x[i]);
}

__global__ void k_half_sqrt(const double* __restrict__ x, int64_t n, double* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = ph::half_sqrt(x[i]);
}

// FP64 pipe throughput probe: every thread runs kPeakChains independent
// chains x <- x m + b (one DFMA each), so the pipe never waits on a result;
// m and b come in as arguments (nothing folds at compile time) and keep the
// iterates bounded (|m| < 1).  Each thread stores its sum, so no chain is
// dead code.
constexpr int kPeakChains = 16;

__global__ void __launch_bounds__(256) k_dfma_peak(int64_t iters, double m, double b, double* __restrict__ sink) {
  double x[kPeakChains];
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) x[j] = (double)(threadIdx.x + j);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) x[j] = fma(x[j], m, b);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) s += x[j];
  sink[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}
}  // namespace

extern "C" ph_status ph_test_fail_alloc(int64_t after) {
  ph::g_fail_alloc_after.store(after < 0 ? -1 : after);
  return PH_OK;
}

extern "C" ph_status ph_test_scan_withhold(int on) {
  ph::g_scan_withhold.store(on ? 1 : 0);
  return PH_OK;
}

extern "C" ph_status ph_pool_in_use(int64_t* bytes) {
  if (!bytes) return PH_ERR_ARG;
  *bytes = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  cudaMemPool_t pool;
  if (e == cudaSuccess) e = ph::pool_for(dev, &pool);
  uint64_t used = 0;
  if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used);
  if (e != cudaSuccess) return ph::cuda_status(e, "ph_pool_in_use");
  *bytes = (int64_t)used;
  return PH_OK;
}

extern "C" ph_status ph_fp64_peak(int64_t iters, double* ops_per_s, double* ms_out, void* stream) {
  if (iters <= 0 || !ops_per_s) return PH_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return ph::cuda_status(e, "ph_fp64_peak");
  constexpr int kThreadsPeak = 256, kBlocksPerSm = 8;
  const unsigned grid = (unsigned)(sms * kBlocksPerSm);
  double* sink = nullptr;
  e = ph::alloc(&sink, (size_t)grid * kThreadsPeak, s);
  if (e != cudaSuccess) return ph::cuda_status(e, "ph_fp64_peak alloc");
  cudaEvent_t a = nullptr, b = nullptr;
  e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = cudaEventRecord(a, s);
  if (e == cudaSuccess) {
    k_dfma_peak<<<grid, kThreadsPeak, 0, s>>>(iters, 0.999999, 1e-3, sink);
    e = ph::launched();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  ph::free_async(sink, s);
  if (e != cudaSuccess) return ph::cuda_status(e, "ph_fp64_peak");
  const double ops = (double)grid * kThreadsPeak * kPeakChains * (double)iters;
  *ops_per_s = ops / (t * 1e-3);
  if (ms_out) *ms_out = t;
  return PH_OK;
}

extern "C" ph_status ph_rcp(const double* x, int64_t n, double* y, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return PH_ERR_ARG;
  if (n == 0) return PH_OK;
  k_rcp<<<ph::grid_for(n), ph::kThreads, 0, (cudaStream_t)stream>>>(x, n, y);
  return ph::cuda_status(ph::launched(), "k_rcp");
}

extern "C" ph_status ph_half_sqrt(const double* x, int64_t n, double* y, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return PH_ERR_ARG;
  if (n == 0) return PH_OK;
  k_half_sqrt<<<ph::grid_for(n), ph::kThreads, 0, (cudaStream_t)stream>>>(x, n, y);
  return ph::cuda_status(ph::launched(), "k_half_sqrt");
}
