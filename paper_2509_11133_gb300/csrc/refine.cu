// Uniform 1 -> 12 refinement on the device (Section 3.4, Listing RedRefine)
// with the edge numbering of Listing NumEdges.
//
// Edges: every local edge of every tet (local order IJ, IK, IL, JK, JL, KL) is a
// key (lo, hi) counting-sorted into buckets by hi; within a bucket each
// occurrence finds the smallest slot 6t+j with the same key (its edge's first
// occurrence).  Edge ids are first-occurrence ranks, as the listing's stable
// unique gives them.  New nodes are numbered as the listing's stable unique of
// [centroid, M1..M6] per tet gives them: walking the tets in order, each tet
// adds its centroid and then the midpoints of its not-yet-seen edges, i.e.
//     centroid(t)        = nC + t + (first occurrences in tets < t),
//     midpoint(edge, f)  = nC + t_f + 1 + (first occurrences before slot f),
// f the edge's first slot.  Coordinates: ((P0 + P1) + P2 + P3) / 4 and
// (P_a + P_b) / 2 with the endpoints of the first occurrence.  Child 1 of
// parent t replaces it; children 2..12 sit at nE + 11 t + (0..10).  Boundary
// triples [n1 n2 n3] (the paper's Db, Nb) become [n1 m12 m13] in place and
// [n2 m23 m12], [n3 m13 m23], [m12 m23 m13] at nF + 3 i + (0..2) (refineFaces).
#include <math.h>
#include <string.h>

#include "edges.cuh"
#include "ph_internal.cuh"

namespace {

// per tet: centroid and midpoint ids, coordinates, the 12 children, and the
// midpoint id of every slot (for the boundary lists)
__global__ void k_refine_tets(const double* __restrict__ coord, const int4* __restrict__ tet, int64_t nE,
                              int64_t nC, const int32_t* __restrict__ first, const int32_t* __restrict__ ebase,
                              double* __restrict__ coord_out, int4* __restrict__ tet_out,
                              int32_t* __restrict__ mid_of_slot) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nE) return;
  const int4 v = tet[t];
  const int cent = (int)(nC + t + ebase[t]);
  int mid[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const int f = first[6 * t + j];
    const int64_t tf = f / 6;
    const int jf = f % 6;
    mid[j] = (int)(nC + tf + 1 + ebase[tf] + rank_in_tet(first, tf, jf));
    mid_of_slot[6 * t + j] = mid[j];
    if (f == (int)(6 * t + j)) {
      int p, q;
      local_edge(j, p, q);
      const double* A = coord + 3 * (int64_t)vget(v, p);
      const double* B = coord + 3 * (int64_t)vget(v, q);
#pragma unroll
      for (int d = 0; d < 3; ++d) coord_out[3 * (int64_t)mid[j] + d] = (A[d] + B[d]) / 2.0;
    }
  }
  const double* P0 = coord + 3 * (int64_t)v.x;
  const double* P1 = coord + 3 * (int64_t)v.y;
  const double* P2 = coord + 3 * (int64_t)v.z;
  const double* P3 = coord + 3 * (int64_t)v.w;
#pragma unroll
  for (int d = 0; d < 3; ++d) coord_out[3 * (int64_t)cent + d] = (((P0[d] + P1[d]) + P2[d]) + P3[d]) / 4.0;
  const int I = v.x, J = v.y, K = v.z, L = v.w;
  const int IJ = mid[0], IK = mid[1], IL = mid[2], JK = mid[3], JL = mid[4], KL = mid[5], C = cent;
  tet_out[t] = make_int4(I, IJ, IK, IL);
  int4* o = tet_out + nE + 11 * t;
  o[0] = make_int4(J, JK, IJ, JL);
  o[1] = make_int4(K, IK, JK, KL);
  o[2] = make_int4(L, KL, JL, IL);
  o[3] = make_int4(IJ, IK, IL, C);
  o[4] = make_int4(JK, IJ, JL, C);
  o[5] = make_int4(IK, JK, KL, C);
  o[6] = make_int4(KL, JL, IL, C);
  o[7] = make_int4(IJ, JK, IK, C);
  o[8] = make_int4(IK, KL, IL, C);
  o[9] = make_int4(IJ, IL, JL, C);
  o[10] = make_int4(KL, JK, JL, C);
}

__device__ __forceinline__ int find_mid(const int2* __restrict__ entries, const int32_t* __restrict__ start,
                                        const int32_t* __restrict__ mid_of_slot, int x, int y, int64_t nC) {
  if (x < 0 || y < 0 || x >= nC || y >= nC || x == y) return -1;
  const int hi = max(x, y), lo = min(x, y);
  for (int k = start[hi]; k < start[hi + 1]; ++k)
    if (entries[k].x == lo) return mid_of_slot[entries[k].y];
  return -1;
}

__global__ void k_refine_lists(const int32_t* __restrict__ in, int64_t nl, const int2* __restrict__ entries,
                               const int32_t* __restrict__ start, const int32_t* __restrict__ mid_of_slot,
                               int64_t nC, int32_t* __restrict__ out, unsigned* status) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nl) return;
  const int n1 = in[3 * i], n2 = in[3 * i + 1], n3 = in[3 * i + 2];
  const int m12 = find_mid(entries, start, mid_of_slot, n1, n2, nC);
  const int m13 = find_mid(entries, start, mid_of_slot, n1, n3, nC);
  const int m23 = find_mid(entries, start, mid_of_slot, n2, n3, nC);
  if (m12 < 0 || m13 < 0 || m23 < 0) { ph_flag(status, PH_ERR_ARG); return; }
  int32_t* a = out + 3 * i;
  a[0] = n1; a[1] = m12; a[2] = m13;
  int32_t* b = out + 3 * (nl + 3 * i);
  b[0] = n2; b[1] = m23; b[2] = m12;
  b[3] = n3; b[4] = m13; b[5] = m23;
  b[6] = m12; b[7] = m23; b[8] = m13;
}

}  // namespace

using namespace ph;

struct ph_refined {
  int64_t nC, nE, nEd, nl;  // refined counts (nEd: edges of the parent mesh)
  double* coord;
  int4* tet;
  int32_t* lists;
};

extern "C" ph_status ph_refine(const double* coord, int64_t nC, const int32_t* tet, int64_t nE,
                               const int32_t* lists, int64_t nl, void* stream, ph_refined** out) {
  if (!out) return PH_ERR_ARG;
  *out = nullptr;
  if (nC < 0 || nE < 0 || nl < 0 || (nE > 0 && (!coord || !tet)) || (nl > 0 && !lists)) return PH_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(tet) & 15u) != 0) return PH_ERR_ARG;  // read as int4
  if (6 * nE >= ((int64_t)1 << 31) - 1 || 12 * nE >= ((int64_t)1 << 31) - 1 || 4 * nl >= ((int64_t)1 << 31) / 3)
    return PH_ERR_OVERFLOW;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nent = 6 * nE;
  int32_t* mid_of_slot = nullptr;
  EdgeNumbering E;
  int64_t* d_tot = nullptr;
  unsigned* status = nullptr;
  ph_refined* r = new ph_refined();
  memset(r, 0, sizeof *r);
  int64_t tot = 0;
  unsigned bits = 0;
  cudaError_t e = cudaSuccess;
  ph_status st = PH_OK;
#define RF_CU(expr)                      \
  do {                                   \
    e = (expr);                          \
    if (e != cudaSuccess) goto cuda_fail; \
  } while (0)
  RF_CU(alloc(&status, 1, s));
  RF_CU(cudaMemsetAsync(status, 0, sizeof(unsigned), s));
  RF_CU(alloc(&d_tot, 1, s));
  st = enqueue_edges(reinterpret_cast<const int4*>(tet), nE, nC, status, d_tot, s, &E);
  if (st != PH_OK) goto fail;
  RF_CU(cudaMemcpyAsync(&tot, d_tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  RF_CU(cudaMemcpyAsync(&bits, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  RF_CU(cudaStreamSynchronize(s));
  if (bits) { st = status_from_bits(bits); goto fail; }
  r->nEd = tot;
  r->nC = nC + nE + tot;
  r->nE = 12 * nE;
  r->nl = 4 * nl;
  if (r->nC >= ((int64_t)1 << 31) - 1) { st = PH_ERR_OVERFLOW; goto fail; }
  RF_CU(alloc(&r->coord, (size_t)(3 * r->nC), s));
  RF_CU(alloc(&r->tet, (size_t)r->nE, s));
  RF_CU(alloc(&r->lists, (size_t)(3 * r->nl), s));
  RF_CU(alloc(&mid_of_slot, (size_t)nent, s));
  if (nC > 0) RF_CU(cudaMemcpyAsync(r->coord, coord, sizeof(double) * 3 * nC, cudaMemcpyDeviceToDevice, s));
  if (nE > 0) {
    k_refine_tets<<<grid_for(nE), kThreads, 0, s>>>(coord, reinterpret_cast<const int4*>(tet), nE, nC, E.first, E.ebase,
                                                    r->coord, r->tet, mid_of_slot);
    RF_CU(launched());
  }
  if (nl > 0) {
    k_refine_lists<<<grid_for(nl), kThreads, 0, s>>>(lists, nl, E.entries, E.start, mid_of_slot, nC, r->lists,
                                                     status);
    RF_CU(launched());
  }
  RF_CU(cudaMemcpyAsync(&bits, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  RF_CU(cudaStreamSynchronize(s));
  if (bits) { st = status_from_bits(bits); goto fail; }
  release_edges(E, s);
  free_async(mid_of_slot, s);
  free_async(d_tot, s);
  free_async(status, s);
  *out = r;
  return PH_OK;
cuda_fail:
  st = cuda_status(e, "ph_refine");
fail:
  release_edges(E, s);
  free_async(mid_of_slot, s);
  free_async(d_tot, s);
  free_async(status, s);
  free_async(r->coord, s);
  free_async(r->tet, s);
  free_async(r->lists, s);
  delete r;
  return st;
#undef RF_CU
}

extern "C" ph_status ph_refined_info(const ph_refined* r, int64_t* nC, int64_t* nE, int64_t* nEd_parent,
                                     int64_t* nl) {
  if (!r) return PH_ERR_ARG;
  if (nC) *nC = r->nC;
  if (nE) *nE = r->nE;
  if (nEd_parent) *nEd_parent = r->nEd;
  if (nl) *nl = r->nl;
  return PH_OK;
}

extern "C" ph_status ph_refined_copy(const ph_refined* r, double* coord, int32_t* tet, int32_t* lists, void* stream) {
  if (!r) return PH_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (coord && r->nC) e = cudaMemcpyAsync(coord, r->coord, sizeof(double) * 3 * r->nC, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && tet && r->nE)
    e = cudaMemcpyAsync(tet, r->tet, sizeof(int4) * r->nE, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && lists && r->nl)
    e = cudaMemcpyAsync(lists, r->lists, sizeof(int32_t) * 3 * r->nl, cudaMemcpyDeviceToDevice, s);
  return cuda_status(e, "ph_refined_copy");
}

extern "C" ph_status ph_refined_destroy(ph_refined* r, void* stream) {
  if (!r) return PH_OK;
  cudaStream_t s = (cudaStream_t)stream;
  free_async(r->coord, s);
  free_async(r->tet, s);
  free_async(r->lists, s);
  delete r;
  return PH_OK;
}
