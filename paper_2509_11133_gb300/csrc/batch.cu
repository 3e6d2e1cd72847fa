// Batched assembly: many problems (meshes of uneven size, each with its own
// coefficient field) assembled and condensed by one persistent kernel.
//
// The elements of all problems are cut into tiles of `tile` consecutive
// elements of one problem (a tile never straddles two problems).  A grid of
// (blocks per SM x SMs) blocks walks the tile table round-robin; each block
// runs the plain path's per-element code (assemble_element) on the tile's
// elements, so every problem's values, rhs and factor are bit-identical to a
// plain ph_assemble call.  The entries that receive atomic contributions are
// cleared first by one batched zero kernel.  The tile size and block shape come
// from ph_batch_autotune, which times candidate configurations on the bound
// problems; the two launches can be instantiated once as a CUDA graph.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "element.cuh"
#include "ph_internal.cuh"

using namespace ph_elem;

namespace {

struct ProbDesc {
  const double* geo;
  const int4* tface;
  const int4* tmult;
  const int4* tpos;
  const ushort4* trel;
  const double* area;
  const int32_t* rowdiag;
  int64_t nE, L;
  const double* a;
  const double* f;
  const double* uD;
  const double* gN;
  double* values;
  double* rhs;
  double* factor;
  unsigned* status;
  double c20, six_over_c;
  int flags;  // bit 0: u_D, bit 1: g_N, bit 2: factor
  int pad;
  const double* lambda;  // recovery (ph_batch_bind_recovery): face values in,
  double* u;             // element values out
};

struct Tile {
  int32_t prob;
  int32_t count;
  int64_t start;
};

template <bool UD, bool GN, bool FAC>
__device__ __forceinline__ void run_tile(const ProbDesc& d, int64_t start, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x)
    assemble_element<UD, GN, FAC>(start + i, d.geo, d.tface, d.tmult, d.tpos, d.trel, d.area, d.a, d.c20,
                                  d.six_over_c, d.f, d.uD, d.gN, d.values, d.rhs, d.factor, d.status);
}

// persistent: block b takes tiles b, b + gridDim.x, ...
__global__ void k_batch_assemble(const ProbDesc* __restrict__ probs, const Tile* __restrict__ tiles, int64_t ntiles) {
  for (int64_t k = blockIdx.x; k < ntiles; k += gridDim.x) {
    const Tile tl = tiles[k];
    const ProbDesc& d = probs[tl.prob];
    switch (d.flags) {  // uniform across the block
      case 0: run_tile<false, false, false>(d, tl.start, tl.count); break;
      case 1: run_tile<true, false, false>(d, tl.start, tl.count); break;
      case 2: run_tile<false, true, false>(d, tl.start, tl.count); break;
      case 3: run_tile<true, true, false>(d, tl.start, tl.count); break;
      case 4: run_tile<false, false, true>(d, tl.start, tl.count); break;
      case 5: run_tile<true, false, true>(d, tl.start, tl.count); break;
      case 6: run_tile<false, true, true>(d, tl.start, tl.count); break;
      default: run_tile<true, true, true>(d, tl.start, tl.count); break;
    }
  }
}

// persistent recovery from the element factor: the same tiles, each problem's
// elements through the plain path's per-element code (recover_element_factored)
__global__ void k_batch_recover(const ProbDesc* __restrict__ probs, const Tile* __restrict__ tiles, int64_t ntiles) {
  for (int64_t k = blockIdx.x; k < ntiles; k += gridDim.x) {
    const Tile tl = tiles[k];
    const ProbDesc& d = probs[tl.prob];
    if (!d.u) continue;
    for (int i = threadIdx.x; i < tl.count; i += blockDim.x) {
      if (d.flags & 2)
        recover_element_factored<true>(tl.start + i, d.geo, d.tface, d.tmult, d.area, d.factor, d.six_over_c, d.f,
                                       d.gN, d.lambda, d.u);
      else
        recover_element_factored<false>(tl.start + i, d.geo, d.tface, d.tmult, d.area, d.factor, d.six_over_c, d.f,
                                        d.gN, d.lambda, d.u);
    }
  }
}

// rhs = 0 and the diagonal of every row = 0, for all problems (row offsets
// of the problems are the exclusive prefix sums roff)
__global__ void k_batch_zero(const ProbDesc* __restrict__ probs, const int64_t* __restrict__ roff, int32_t nprob,
                             int64_t nrows) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nrows; g += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nprob - 1;  // problem of row g: last roff[p] <= g
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (roff[mid] <= g) lo = mid; else hi = mid - 1;
    }
    const ProbDesc& d = probs[lo];
    const int64_t l = g - roff[lo];
    d.rhs[l] = 0.0;
    d.values[d.rowdiag[l]] = 0.0;
  }
}

}  // namespace

struct ph_batch {
  int device;
  int32_t n;
  std::vector<const ph_mesh*> meshes;
  std::vector<ProbDesc> host;
  ProbDesc* d_probs;
  int64_t* d_roff;
  int64_t nrows, nelems;
  Tile* d_tiles;
  int64_t ntiles;
  int32_t tile, threads, blocks_per_sm, sms;
  bool bound, recover;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
};

using namespace ph;

static void drop_graph(ph_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// (Re)build the tile table for b->tile.
static ph_status build_tiles(ph_batch* b, cudaStream_t s) {
  std::vector<Tile> t;
  for (int32_t p = 0; p < b->n; ++p) {
    const int64_t nE = b->meshes[p]->nE;
    for (int64_t st = 0; st < nE; st += b->tile)
      t.push_back(Tile{p, (int32_t)std::min<int64_t>(b->tile, nE - st), st});
  }
  free_async(b->d_tiles, s);
  b->d_tiles = nullptr;
  b->ntiles = (int64_t)t.size();
  cudaError_t e = alloc(&b->d_tiles, t.size(), s);
  if (e == cudaSuccess && !t.empty())
    e = cudaMemcpyAsync(b->d_tiles, t.data(), sizeof(Tile) * t.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // t is a host temporary
  drop_graph(b);
  return cuda_status(e, "ph_batch tiles");
}

extern "C" ph_status ph_batch_create(ph_mesh* const* meshes, int32_t n, void* stream, ph_batch** out) {
  if (!out || n < 0 || (n > 0 && !meshes)) return PH_ERR_ARG;
  *out = nullptr;
  for (int32_t i = 0; i < n; ++i) {
    if (!meshes[i]) return PH_ERR_ARG;
    if (meshes[i]->geo_dw) {  // the batched kernel runs the fp64 element code
      set_error_text("ph_batch_create: a mesh holds a double-word geometry record (ph_mesh_create_dw)");
      return PH_ERR_ARG;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  ph_batch* b = new ph_batch();
  b->n = n;
  b->meshes.assign(meshes, meshes + n);
  b->host.resize(n);
  b->d_probs = nullptr;
  b->d_roff = nullptr;
  b->d_tiles = nullptr;
  b->graph = nullptr;
  b->exec = nullptr;
  b->bound = false;
  b->recover = false;
  b->tile = 1024;
  b->threads = 128;
  b->blocks_per_sm = 4;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
  std::vector<int64_t> roff(n + 1, 0);
  b->nelems = 0;
  for (int32_t i = 0; i < n; ++i) {
    roff[i + 1] = roff[i] + meshes[i]->L;
    b->nelems += meshes[i]->nE;
    if (meshes[i]->device != b->device) e = cudaErrorInvalidDevice;
  }
  b->nrows = roff[n];
  if (e == cudaSuccess) e = alloc(&b->d_probs, (size_t)std::max(n, 1), s);
  if (e == cudaSuccess) e = alloc(&b->d_roff, (size_t)n + 1, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_roff, roff.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  ph_status st = cuda_status(e, "ph_batch_create");
  if (st == PH_OK) st = build_tiles(b, s);
  if (st != PH_OK) {
    free_async(b->d_probs, s);
    free_async(b->d_roff, s);
    free_async(b->d_tiles, s);
    delete b;
    return st;
  }
  *out = b;
  return PH_OK;
}

extern "C" ph_status ph_batch_destroy(ph_batch* b, void* stream) {
  if (!b) return PH_OK;
  cudaStream_t s = (cudaStream_t)stream;
  drop_graph(b);
  free_async(b->d_probs, s);
  free_async(b->d_roff, s);
  free_async(b->d_tiles, s);
  delete b;
  return PH_OK;
}

extern "C" ph_status ph_batch_bind(ph_batch* b, const double* const* a, const double* c, const double* const* f_face,
                                   const double* const* uD_face, const double* const* gN_face,
                                   double* const* values, double* const* rhs, double* const* factor, void* stream) {
  if (!b || (b->n > 0 && (!a || !c || !f_face || !values || !rhs))) return PH_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  for (int32_t i = 0; i < b->n; ++i) {
    const ph_mesh* m = b->meshes[i];
    if (!(c[i] > 0.0) || !(c[i] < INFINITY)) return PH_ERR_ARG;
    if (m->nE > 0 && (!a[i] || !f_face[i])) return PH_ERR_ARG;
    if ((m->nnz > 0 && !values[i]) || (m->L > 0 && !rhs[i])) return PH_ERR_ARG;
    if (b->recover && b->host[i].u && (!factor || !factor[i])) return PH_ERR_ARG;  // recovery reads the factor
  }
  for (int32_t i = 0; i < b->n; ++i) {
    const ph_mesh* m = b->meshes[i];
    ProbDesc& d = b->host[i];
    const double* keep_lambda = d.lambda;  // recovery arrays survive a rebind
    double* keep_u = d.u;
    memset(&d, 0, sizeof d);
    d.lambda = keep_lambda;
    d.u = keep_u;
    d.geo = m->geo;
    d.tface = m->tface;
    d.tmult = m->tmult;
    d.tpos = m->tpos;
    d.trel = m->trel;
    d.area = m->face_area;
    d.rowdiag = m->rowdiag;
    d.nE = m->nE;
    d.L = m->L;
    d.a = a[i];
    d.f = f_face[i];
    d.uD = uD_face ? uD_face[i] : nullptr;
    d.gN = gN_face ? gN_face[i] : nullptr;
    d.values = values[i];
    d.rhs = rhs[i];
    d.factor = factor ? factor[i] : nullptr;
    d.status = m->status;
    d.c20 = c[i] / 20.0;
    d.six_over_c = 6.0 / c[i];
    d.flags = ((d.uD && m->nFd > 0) ? 1 : 0) | ((d.gN && m->nFn > 0) ? 2 : 0) | (d.factor ? 4 : 0);
  }
  cudaError_t e = cudaSuccess;
  if (b->n > 0)
    e = cudaMemcpyAsync(b->d_probs, b->host.data(), sizeof(ProbDesc) * b->n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host copy may change after return
  if (e != cudaSuccess) return cuda_status(e, "ph_batch_bind");
  b->bound = true;
  return PH_OK;
}

static cudaError_t launch_batch(ph_batch* b, cudaStream_t s) {
  if (b->nrows > 0) {
    const unsigned zg = (unsigned)std::min<int64_t>((b->nrows + 255) / 256, (int64_t)b->sms * 8);
    k_batch_zero<<<zg, 256, 0, s>>>(b->d_probs, b->d_roff, b->n, b->nrows);
    cudaError_t e = launched();
    if (e != cudaSuccess) return e;
  }
  if (b->ntiles > 0) {
    const unsigned grid = (unsigned)std::min<int64_t>(b->ntiles, (int64_t)b->sms * b->blocks_per_sm);
    k_batch_assemble<<<grid, b->threads, 0, s>>>(b->d_probs, b->d_tiles, b->ntiles);
    cudaError_t e = launched();
    if (e != cudaSuccess || !b->recover) return e;
    k_batch_recover<<<grid, b->threads, 0, s>>>(b->d_probs, b->d_tiles, b->ntiles);
    return launched();
  }
  return cudaSuccess;
}

static int batch_launches(const ph_batch* b) {
  return (b->nrows > 0 ? 1 : 0) + (b->ntiles > 0 ? (b->recover ? 2 : 1) : 0);
}

extern "C" ph_status ph_batch_assemble(ph_batch* b, void* stream) {
  if (!b || !b->bound) return PH_ERR_ARG;
  return cuda_status(launch_batch(b, (cudaStream_t)stream), "ph_batch_assemble");
}

extern "C" ph_status ph_batch_set_config(ph_batch* b, int32_t tile, int32_t threads, int32_t blocks_per_sm,
                                         void* stream) {
  if (!b || tile < 32 || threads < 32 || threads > 1024 || threads % 32 || blocks_per_sm < 1 || blocks_per_sm > 32)
    return PH_ERR_ARG;
  b->threads = threads;
  b->blocks_per_sm = blocks_per_sm;
  drop_graph(b);
  if (tile != b->tile) {
    b->tile = tile;
    return build_tiles(b, (cudaStream_t)stream);
  }
  return PH_OK;
}

extern "C" ph_status ph_batch_get_config(const ph_batch* b, int32_t* tile, int32_t* threads, int32_t* blocks_per_sm) {
  if (!b) return PH_ERR_ARG;
  if (tile) *tile = b->tile;
  if (threads) *threads = b->threads;
  if (blocks_per_sm) *blocks_per_sm = b->blocks_per_sm;
  return PH_OK;
}

extern "C" ph_status ph_batch_autotune(ph_batch* b, int32_t reps, float* best_ms, void* stream) {
  if (!b || !b->bound || reps < 1) return PH_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  static const int32_t tiles[] = {256, 1024, 4096, 16384};
  static const int32_t threads[] = {64, 128, 256};
  static const int32_t bps[] = {2, 4, 8};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 1e30f;
  int32_t bt = b->tile, bth = b->threads, bb = b->blocks_per_sm;
  for (int32_t tl : tiles) {
    if (e != cudaSuccess) break;
    ph_status st = ph_batch_set_config(b, tl, b->threads, b->blocks_per_sm, stream);
    if (st != PH_OK) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return st;
    }
    for (int32_t th : threads)
      for (int32_t bp : bps) {
        if (e != cudaSuccess) break;
        b->threads = th;
        b->blocks_per_sm = bp;
        e = launch_batch(b, s);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        for (int32_t r = 0; r < reps && e == cudaSuccess; ++r) e = launch_batch(b, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        ms /= (float)reps;
        if (e == cudaSuccess && ms < best) {
          best = ms;
          bt = tl;
          bth = th;
          bb = bp;
        }
      }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_status(e, "ph_batch_autotune");
  if (best_ms) *best_ms = best;
  return ph_batch_set_config(b, bt, bth, bb, stream);
}

extern "C" ph_status ph_batch_graph_launch(ph_batch* b, void* stream) {
  if (!b || !b->bound) return PH_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (!b->exec) {
    // capture the two launches on a private stream and instantiate once
    cudaStream_t cs = nullptr;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const int64_t before = g_launches.load();
      cudaError_t le = launch_batch(b, cs);
      g_launches.store(before);  // recorded, not run: counted at each graph launch
      e = cudaStreamEndCapture(cs, &b->graph);
      if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      drop_graph(b);
      return cuda_status(e, "ph_batch_graph_launch capture");
    }
  }
  e = cudaGraphLaunch(b->exec, s);
  if (e == cudaSuccess) g_launches.fetch_add(batch_launches(b), std::memory_order_relaxed);
  return cuda_status(e, "ph_batch_graph_launch");
}

extern "C" ph_status ph_batch_bind_recovery(ph_batch* b, const double* const* lambda, double* const* u,
                                            void* stream) {
  if (!b || !b->bound) return PH_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const bool on = lambda != nullptr;
  for (int32_t i = 0; i < b->n && on; ++i) {
    const ph_mesh* m = b->meshes[i];
    if (m->nE > 0 && (!u || !u[i] || !b->host[i].factor || (m->L > 0 && !lambda[i]))) return PH_ERR_ARG;
  }
  for (int32_t i = 0; i < b->n; ++i) {
    b->host[i].lambda = on ? lambda[i] : nullptr;
    b->host[i].u = on ? u[i] : nullptr;
  }
  cudaError_t e = cudaSuccess;
  if (b->n > 0)
    e = cudaMemcpyAsync(b->d_probs, b->host.data(), sizeof(ProbDesc) * b->n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e, "ph_batch_bind_recovery");
  if (on != b->recover) drop_graph(b);  // the graph gains or loses the recovery launch
  b->recover = on;
  return PH_OK;
}
