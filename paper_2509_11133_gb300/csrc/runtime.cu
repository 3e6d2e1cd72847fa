// Runtime pieces of the library: status strings, error messages, launch
// counter, the stream-ordered memory pool and a device-wide exclusive scan.
#include <stdio.h>
#include <string.h>

#include <mutex>

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
    g_pool_ok[dev] = true;
  }
  *out = g_pools[dev];
  return cudaSuccess;
}

cudaError_t alloc_bytes(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
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
constexpr int SCAN_I = 8;
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

__global__ void k_scan_reduce(const int32_t* __restrict__ in, int64_t n, int64_t* __restrict__ tile_sums) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_I; ++i) {
    int64_t idx = base + (int64_t)i * SCAN_T + threadIdx.x;
    if (idx < n) s += in[idx];
  }
  int64_t tot;
  block_excl_scan<int64_t, SCAN_T>(s, &tot);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// One block: exclusive scan of the tile sums in place; total to *d_total.
__global__ void k_scan_tiles(int64_t* __restrict__ tile_sums, int64_t ntiles, int64_t* __restrict__ d_total) {
  int64_t carry = 0;
  for (int64_t base = 0; base < ntiles; base += 1024) {
    int64_t idx = base + threadIdx.x;
    int64_t v = idx < ntiles ? tile_sums[idx] : 0;
    int64_t tot;
    int64_t ex = block_excl_scan<int64_t, 1024>(v, &tot);
    if (idx < ntiles) tile_sums[idx] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *d_total = carry;
}

__global__ void k_scan_apply(const int32_t* in, int32_t* out, int64_t n, const int64_t* __restrict__ tile_offs) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_I;
  int32_t v[SCAN_I];
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_I; ++i) {
    int64_t idx = base + i;
    v[i] = idx < n ? in[idx] : 0;
    s += v[i];
  }
  int64_t tot;
  int64_t run = tile_offs[blockIdx.x] + block_excl_scan<int64_t, SCAN_T>(s, &tot);
#pragma unroll
  for (int i = 0; i < SCAN_I; ++i) {
    int64_t idx = base + i;
    if (idx < n) out[idx] = (int32_t)run;
    run += v[i];
  }
}

ph_status exclusive_scan(const int32_t* in, int32_t* out, int64_t n, int64_t* d_total, cudaStream_t s) {
  int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (ntiles < 1) ntiles = 1;
  int64_t* tiles = nullptr;
  cudaError_t e = alloc(&tiles, (size_t)ntiles, s);
  if (e != cudaSuccess) return cuda_status(e, "scan alloc");
  k_scan_reduce<<<(unsigned)ntiles, SCAN_T, 0, s>>>(in, n, tiles);
  e = launched();
  if (e == cudaSuccess) {
    k_scan_tiles<<<1, 1024, 0, s>>>(tiles, ntiles, d_total);
    e = launched();
  }
  if (e == cudaSuccess) {
    k_scan_apply<<<(unsigned)ntiles, SCAN_T, 0, s>>>(in, out, n, tiles);
    e = launched();
  }
  free_async(tiles, s);
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

namespace {
__global__ void k_rcp(const double* __restrict__ x, int64_t n, double* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = ph::rcp_newton(x[i]);
}
}  // namespace

extern "C" ph_status ph_rcp(const double* x, int64_t n, double* y, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return PH_ERR_ARG;
  if (n == 0) return PH_OK;
  k_rcp<<<ph::grid_for(n), ph::kThreads, 0, (cudaStream_t)stream>>>(x, n, y);
  return ph::cuda_status(ph::launched(), "k_rcp");
}
