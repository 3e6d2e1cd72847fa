// Edge numbering of Listing NumEdges on the device, shared by the refinement
// (ph_refine) and the edge-patch Schwarz preconditioner (ph_schwarz_*).
//
// Every local edge of every tet (local order IJ, IK, IL, JK, JL, KL; slot
// 6t+j) is a key (lo, hi) counting-sorted into buckets by hi; within a bucket
// each occurrence finds the smallest slot with the same key (its edge's first
// occurrence).  Edge ids are first-occurrence ranks, as the listing's stable
// unique gives them: edge_id(slot) = ebase[t_f] + (first occurrences before
// slot f inside tet t_f), f = first[slot].
#pragma once

#include "ph_internal.cuh"

namespace {  // device code: a private copy per translation unit

__device__ __forceinline__ int vget(int4 v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }

// local edge j: IJ, IK, IL, JK, JL, KL
__device__ __forceinline__ void local_edge(int j, int& p, int& q) {
  const int P[6] = {0, 0, 0, 1, 1, 2};
  const int Q[6] = {1, 2, 3, 2, 3, 3};
  p = P[j];
  q = Q[j];
}

__device__ __forceinline__ bool valid_tet(int4 v, int64_t nC) {
  bool in = v.x >= 0 && v.y >= 0 && v.z >= 0 && v.w >= 0 && v.x < nC && v.y < nC && v.z < nC && v.w < nC;
  bool distinct = v.x != v.y && v.x != v.z && v.x != v.w && v.y != v.z && v.y != v.w && v.z != v.w;
  return in && distinct;
}

__global__ void k_edge_count(const int4* __restrict__ tet, int64_t nE, int64_t nC, int32_t* __restrict__ cnt,
                             unsigned* status) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nE) return;
  const int4 v = tet[t];
  if (!valid_tet(v, nC)) { ph_flag(status, PH_ERR_ARG); return; }
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    int p, q;
    local_edge(j, p, q);
    atomicAdd(&cnt[max(vget(v, p), vget(v, q))], 1);
  }
}

// entry = (lo, slot)
// Both kernels below return at once once an invalid tet was flagged: the
// entries of such a mesh are incomplete and must not be dereferenced.
__global__ void k_edge_fill(const int4* __restrict__ tet, int64_t nE, int64_t nC, const int32_t* __restrict__ start,
                            int32_t* __restrict__ cnt, int2* __restrict__ entries, const unsigned* status) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nE || *status) return;
  const int4 v = tet[t];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    int p, q;
    local_edge(j, p, q);
    const int a = vget(v, p), b = vget(v, q);
    const int hi = max(a, b), lo = min(a, b);
    const int pos = start[hi] + atomicSub(&cnt[hi], 1) - 1;
    entries[pos] = make_int2(lo, (int)(6 * t + j));
  }
}

// first[slot] = smallest slot with the same (lo, hi); the bucket of entry i is
// found from its slot's tet (hi = max of the slot's endpoints).
__global__ void k_edge_first(const int4* __restrict__ tet, const int2* __restrict__ entries, int64_t nent,
                             const int32_t* __restrict__ start, int32_t* __restrict__ first, const unsigned* status) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nent || *status) return;
  const int2 e = entries[i];
  const int t = e.y / 6, j = e.y % 6;
  int p, q;
  local_edge(j, p, q);
  const int4 v = tet[t];
  const int hi = max(vget(v, p), vget(v, q));
  const int lo = start[hi], end = start[hi + 1];
  int m = e.y;
  for (int k = lo; k < end; ++k) {
    const int2 f = entries[k];
    if (f.x == e.x && f.y < m) m = f.y;
  }
  first[e.y] = m;
}

__global__ void k_edge_newcount(const int32_t* __restrict__ first, int64_t nE, int32_t* __restrict__ ecount) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nE) return;
  int c = 0;
#pragma unroll
  for (int j = 0; j < 6; ++j) c += first[6 * t + j] == (int)(6 * t + j);
  ecount[t] = c;
}

// first occurrences before local edge j of tet t (inclusive of tets < t: ebase)
__device__ __forceinline__ int rank_in_tet(const int32_t* __restrict__ first, int64_t t, int j) {
  int r = 0;
  for (int k = 0; k < j; ++k) r += first[6 * t + k] == (int)(6 * t + k);
  return r;
}

// Edge id of a slot from the numbering (first occurrence slot f = first[slot]).
__device__ __forceinline__ int edge_id(const int32_t* __restrict__ first, const int32_t* __restrict__ ebase,
                                       int64_t slot) {
  const int f = first[slot];
  return ebase[f / 6] + rank_in_tet(first, f / 6, f % 6);
}

// Buffers of one numbering (pool memory, stream-ordered).
struct EdgeNumbering {
  int32_t *cnt = nullptr, *start = nullptr, *first = nullptr, *ebase = nullptr;
  int2* entries = nullptr;
};

void release_edges(EdgeNumbering& E, cudaStream_t s) {
  ph::free_async(E.cnt, s);
  ph::free_async(E.start, s);
  ph::free_async(E.entries, s);
  ph::free_async(E.first, s);
  ph::free_async(E.ebase, s);
  E = EdgeNumbering();
}

// Enqueue the numbering of the edges of tet[nE] (vertex ids checked against
// nC; errors go to *status); the edge count lands in *d_nEd.  No
// synchronisation.
ph_status enqueue_edges(const int4* tet, int64_t nE, int64_t nC, unsigned* status, int64_t* d_nEd, cudaStream_t s,
                        EdgeNumbering* E) {
  const int64_t nent = 6 * nE;
  cudaError_t e = ph::alloc(&E->cnt, (size_t)nC + 1, s);
  if (e == cudaSuccess) e = ph::alloc(&E->start, (size_t)nC + 1, s);
  if (e == cudaSuccess) e = ph::alloc(&E->entries, (size_t)nent, s);
  if (e == cudaSuccess) e = ph::alloc(&E->first, (size_t)nent, s);
  if (e == cudaSuccess) e = ph::alloc(&E->ebase, (size_t)nE + 1, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(E->cnt, 0, sizeof(int32_t) * (nC + 1), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(E->ebase, 0, sizeof(int32_t) * (nE + 1), s);
  if (e == cudaSuccess && nE > 0) {
    k_edge_count<<<ph::grid_for(nE), ph::kThreads, 0, s>>>(tet, nE, nC, E->cnt, status);
    e = ph::launched();
  }
  if (e != cudaSuccess) return ph::cuda_status(e, "edge numbering");
  ph_status st = ph::exclusive_scan(E->cnt, E->start, nC + 1, d_nEd, s, status);
  if (st != PH_OK) return st;
  if (nE > 0) {
    k_edge_fill<<<ph::grid_for(nE), ph::kThreads, 0, s>>>(tet, nE, nC, E->start, E->cnt, E->entries, status);
    k_edge_first<<<ph::grid_for(nent), ph::kThreads, 0, s>>>(tet, E->entries, nent, E->start, E->first, status);
    k_edge_newcount<<<ph::grid_for(nE), ph::kThreads, 0, s>>>(E->first, nE, E->ebase);
    e = ph::launched(3);
    if (e != cudaSuccess) return ph::cuda_status(e, "edge numbering");
  }
  return ph::exclusive_scan(E->ebase, E->ebase, nE + 1, d_nEd, s, status);
}

}  // namespace
