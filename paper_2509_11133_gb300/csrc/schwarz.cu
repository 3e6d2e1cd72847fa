// Additive Schwarz preconditioner over edge patches for the condensed system
// H Lambda = rhs (Eq. schur).  H = sum_T d_T d_T' / (c|T|) + (a smaller
// part): the first term penalises each element's flux balance, and its null
// space -- divergence-free face fluxes -- is spanned by fields that live on
// the faces around one edge.  Exact solves on those edge patches,
//     M = sum_e R_e' (R_e H R_e')^-1 R_e,
// take the penalty out of the condition number.
//
// Construction (ph_schwarz_create): edges numbered as Listing NumEdges (the
// shared edge kernels); each face-edge incidence counted once, from the
// face's T+ tet; patch members sorted; each patch block extracted from the
// CSR and inverted in FP64 by Cholesky (upper triangle stored).
// Application (schwarz_apply): one thread per patch computes y_e = block^-1 r_e
// (sums in member order), then one thread per multiplier adds the three
// values of its face's three edges in a fixed order -- no atomics, so a solve
// repeats bit for bit.
#include <math.h>
#include <string.h>

#include "edges.cuh"
#include "pcg.cuh"
#include "ph_internal.cuh"

namespace {

using namespace ph_pcg;

__device__ __forceinline__ int comp4(int4 v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }

// Local faces [abc], [acd], [adb], [dcb] containing local edge j
// (IJ, IK, IL, JK, JL, KL).
__device__ __forceinline__ void faces_of_edge(int j, int& a, int& b) {
  const int A[6] = {0, 0, 1, 0, 2, 1};
  const int B[6] = {2, 1, 2, 3, 3, 3};
  a = A[j];
  b = B[j];
}

// Position of (i, j), i <= j, in a packed row-major upper triangle of order k.
__host__ __device__ __forceinline__ int upper(int i, int j, int k) { return i * k - i * (i - 1) / 2 + (j - i); }

// Incidences per edge (faces with a multiplier, counted from their T+ tet)
// and the edge's vertex pair (written by its first occurrence).
__global__ void k_patch_count(const int4* __restrict__ tet, const int4* __restrict__ tface,
                              const int4* __restrict__ tmult, int64_t nE, const int32_t* __restrict__ first,
                              const int32_t* __restrict__ ebase, int32_t* __restrict__ cnt, int2* __restrict__ ev) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nE) return;
  const int4 v = tet[t], tf = tface[t], tm = tmult[t];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const int64_t slot = 6 * t + j;
    const int e = edge_id(first, ebase, slot);
    if (first[slot] == (int)slot) {
      int p, q;
      local_edge(j, p, q);
      const int x = vget(v, p), y = vget(v, q);
      ev[e] = make_int2(min(x, y), max(x, y));
    }
    int fa, fb;
    faces_of_edge(j, fa, fb);
    if (comp4(tf, fa) >= 0 && comp4(tm, fa) != PH_NO_MULT) atomicAdd(&cnt[e], 1);
    if (comp4(tf, fb) >= 0 && comp4(tm, fb) != PH_NO_MULT) atomicAdd(&cnt[e], 1);
  }
}

__global__ void k_patch_fill(const int4* __restrict__ tface, const int4* __restrict__ tmult, int64_t nE,
                             const int32_t* __restrict__ first, const int32_t* __restrict__ ebase,
                             const int32_t* __restrict__ off, int32_t* __restrict__ fill, int32_t* __restrict__ mem) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nE) return;
  const int4 tf = tface[t], tm = tmult[t];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const int e = edge_id(first, ebase, 6 * t + j);
    int f2[2];
    faces_of_edge(j, f2[0], f2[1]);
#pragma unroll
    for (int u = 0; u < 2; ++u)
      if (comp4(tf, f2[u]) >= 0 && comp4(tm, f2[u]) != PH_NO_MULT)
        mem[off[e] + atomicAdd(&fill[e], 1)] = comp4(tm, f2[u]) & PH_ID_MASK;
  }
}

// Members in ascending order (the fill order is not deterministic) and the
// size of the patch's block storage.
__global__ void k_patch_sort(int64_t nEd, const int32_t* __restrict__ off, int32_t* __restrict__ mem,
                             int32_t* __restrict__ bsize) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nEd) return;
  const int b = off[e], k = off[e + 1] - b;
  for (int i = 1; i < k; ++i) {
    const int x = mem[b + i];
    int j = i - 1;
    while (j >= 0 && mem[b + j] > x) {
      mem[b + j + 1] = mem[b + j];
      --j;
    }
    mem[b + j + 1] = x;
  }
  bsize[e] = k <= kSchwarzDense ? k * (k + 1) / 2 : k;
}

__device__ __forceinline__ double csr_entry(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                                            const double* __restrict__ values, int row, int col) {
  for (int j = rowptr[row]; j < rowptr[row + 1]; ++j)
    if (colind[j] == col) return values[j];
  return 0.0;
}

// Invert each patch block: Cholesky A = G G', then A^-1 = G^-T G^-1 (upper
// triangle stored).  Blocks wider than kSchwarzDense keep 1/diag.
__global__ void k_patch_factor(int64_t nEd, const int32_t* __restrict__ off, const int32_t* __restrict__ mem,
                               const int32_t* __restrict__ boff, const int32_t* __restrict__ rowptr,
                               const int32_t* __restrict__ colind, const double* __restrict__ values,
                               double* __restrict__ blk, unsigned* status) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nEd) return;
  const int b = off[e], k = off[e + 1] - b;
  double* out = blk + boff[e];
  if (k > kSchwarzDense) {
    for (int i = 0; i < k; ++i) {
      const double d = csr_entry(rowptr, colind, values, mem[b + i], mem[b + i]);
      if (!(d > 0.0)) ph_flag(status, PH_ERR_ARG);
      out[i] = d > 0.0 ? 1.0 / d : 0.0;
    }
    return;
  }
  constexpr int K = kSchwarzDense;
  double g[K * K];  // lower Cholesky factor, then its inverse (row-major)
  for (int i = 0; i < k; ++i)
    for (int j = 0; j <= i; ++j) g[i * K + j] = csr_entry(rowptr, colind, values, mem[b + i], mem[b + j]);
  for (int j = 0; j < k; ++j) {
    double d = g[j * K + j];
    for (int m = 0; m < j; ++m) d -= g[j * K + m] * g[j * K + m];
    if (!(d > 0.0)) {
      ph_flag(status, PH_ERR_ARG);
      return;
    }
    const double gj = sqrt(d);
    g[j * K + j] = gj;
    for (int i = j + 1; i < k; ++i) {
      double s = g[i * K + j];
      for (int m = 0; m < j; ++m) s -= g[i * K + m] * g[j * K + m];
      g[i * K + j] = s / gj;
    }
  }
  // G^-1 in place (lower triangular), column by column
  for (int j = 0; j < k; ++j) {
    g[j * K + j] = 1.0 / g[j * K + j];
    for (int i = j + 1; i < k; ++i) {
      double s = 0.0;
      for (int m = j; m < i; ++m) s -= g[i * K + m] * g[m * K + j];
      g[i * K + j] = s / g[i * K + i];
    }
  }
  // A^-1 = G^-T G^-1: (i, j) = sum_{m >= max(i, j)} Gi[m][i] Gi[m][j]
  for (int i = 0; i < k; ++i)
    for (int j = i; j < k; ++j) {
      double s = 0.0;
      for (int m = j; m < k; ++m) s += g[m * K + i] * g[m * K + j];
      out[upper(i, j, k)] = s;
    }
}

__global__ void k_mult_to_face(const int32_t* __restrict__ face_mult, int64_t nF, int32_t* __restrict__ m2f) {
  const int64_t F = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (F < nF && face_mult[F] >= 0) m2f[face_mult[F]] = (int)F;
}

// fslot[3 l + s]: position in mem of multiplier l in the patch of the edge of
// its face opposite the face's vertex s (face_vtx order).
__global__ void k_face_slots(int64_t nEd, const int32_t* __restrict__ off, const int32_t* __restrict__ mem,
                             const int2* __restrict__ ev, const int32_t* __restrict__ m2f,
                             const int32_t* __restrict__ face_vtx, int32_t* __restrict__ fslot) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nEd) return;
  const int2 lh = ev[e];
  for (int i = off[e]; i < off[e + 1]; ++i) {
    const int l = mem[i];
    const int64_t F = m2f[l];
    const int x = face_vtx[3 * F], y = face_vtx[3 * F + 1];
    const int s = (x != lh.x && x != lh.y) ? 0 : (y != lh.x && y != lh.y) ? 1 : 2;
    fslot[3 * (int64_t)l + s] = i;
  }
}

// y_e = block_e^-1 r_e, one thread per patch; registers for patches of at
// most 8 members (all of them on the refined Kuhn meshes).
template <int KMAX>
__device__ __forceinline__ void patch_solve(int b, int k, const double* __restrict__ M, const int32_t* __restrict__ mem,
                                            const double* __restrict__ r, double* __restrict__ y) {
  double rv[KMAX];
#pragma unroll
  for (int j = 0; j < KMAX; ++j) rv[j] = j < k ? __ldg(r + __ldg(mem + b + j)) : 0.0;
#pragma unroll
  for (int i = 0; i < KMAX; ++i) {
    if (i >= k) break;
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
      if (j >= k) break;
      s = fma(__ldg(M + (i <= j ? upper(i, j, k) : upper(j, i, k))), rv[j], s);
    }
    y[b + i] = s;
  }
}

__global__ void __launch_bounds__(256) k_schwarz_patch(int64_t nEd, const int32_t* __restrict__ off,
                                                       const int32_t* __restrict__ mem,
                                                       const int32_t* __restrict__ boff,
                                                       const double* __restrict__ blk, const double* __restrict__ r,
                                                       double* __restrict__ y) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nEd) return;
  const int b = off[e], k = off[e + 1] - b;
  const double* M = blk + boff[e];
  if (k <= 8) {
    patch_solve<8>(b, k, M, mem, r, y);
  } else if (k <= kSchwarzDense) {
    patch_solve<kSchwarzDense>(b, k, M, mem, r, y);
  } else {
    for (int i = 0; i < k; ++i) y[b + i] = M[i] * r[mem[b + i]];
  }
}

// z = sum of the three patch values of each multiplier (fixed order), r.z;
// the last block sets rz (init) or beta = r.z / rz_old and rz.
__global__ void __launch_bounds__(RT) k_schwarz_face(int64_t L, const int32_t* __restrict__ fslot,
                                                     const double* __restrict__ y, const double* __restrict__ r,
                                                     double* __restrict__ z, double* __restrict__ part,
                                                     Scalars* __restrict__ sc, bool init) {
  double rz = 0.0;
  for (int64_t l = blockIdx.x * (int64_t)RT + threadIdx.x; l < L; l += (int64_t)RB * RT) {
    const int s0 = fslot[3 * l], s1 = fslot[3 * l + 1], s2 = fslot[3 * l + 2];
    const double zl = (y[s0] + y[s1]) + y[s2];
    z[l] = zl;
    rz = fma(r[l], zl, rz);
  }
  rz = block_sum(rz);
  if (threadIdx.x == 0) part[RB + blockIdx.x] = rz;
  if (last_block(&sc->done)) {
    const double rz_t = sum_partials(part, RB);
    if (threadIdx.x == 0) {
      if (init) {
        sc->beta = 0.0;
      } else {
        const double rz_old = sc->rz;
        sc->beta = rz_old > 0.0 ? rz_t / rz_old : 0.0;
      }
      sc->rz = rz_t;
      sc->done = 0;
    }
  }
}

}  // namespace

namespace ph_pcg {

cudaError_t schwarz_apply(const ph_schwarz* P, const double* r, double* z, double* y, double* part, Scalars* sc,
                          bool init, cudaStream_t s) {
  if (P->nEd > 0)
    k_schwarz_patch<<<ph::grid_for(P->nEd), 256, 0, s>>>(P->nEd, P->off, P->mem, P->boff, P->blk, r, y);
  k_schwarz_face<<<RB, RT, 0, s>>>(P->L, P->fslot, y, r, z, part, sc, init);
  return ph::launched(P->nEd > 0 ? 2 : 1);
}

}  // namespace ph_pcg

using namespace ph;

static void schwarz_free(ph_schwarz* P, cudaStream_t s) {
  if (!P) return;
  free_async(P->off, s);
  free_async(P->mem, s);
  free_async(P->boff, s);
  free_async(P->blk, s);
  free_async(P->fslot, s);
  delete P;
}

extern "C" ph_status ph_schwarz_create(const ph_mesh* m, const double* values, void* stream, ph_schwarz** out) {
  if (!out) return PH_ERR_ARG;
  *out = nullptr;
  if (!m || (m->nnz > 0 && !values)) return PH_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  ph_schwarz* P = new ph_schwarz();
  memset(P, 0, sizeof *P);
  P->device = m->device;
  P->L = m->L;
  const int64_t nE = m->nE, nF = m->nF, L = m->L;
  EdgeNumbering E;
  int32_t *cnt = nullptr, *fill = nullptr, *bsize = nullptr, *m2f = nullptr;
  int2* ev = nullptr;
  int64_t* d_tot = nullptr;  // [0] nEd, [1] members, [2] block doubles
  unsigned* status = nullptr;
  int64_t tot[3] = {0, 0, 0};
  unsigned bits = 0;
  ph_status st = PH_OK;
  cudaError_t e = alloc(&status, 1, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = alloc(&d_tot, 3, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_tot, 0, 3 * sizeof(int64_t), s);
  if (e != cudaSuccess) { st = cuda_status(e, "ph_schwarz_create"); goto done; }
  st = enqueue_edges(m->tet, nE, m->nC, status, d_tot, s, &E);
  if (st != PH_OK) goto done;
  e = cudaMemcpyAsync(tot, d_tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { st = cuda_status(e, "ph_schwarz_create"); goto done; }
  P->nEd = tot[0];
  if (P->nEd >= ((int64_t)1 << 31) - 1) { st = PH_ERR_OVERFLOW; goto done; }

  // patch members
  e = alloc(&cnt, (size_t)P->nEd + 1, s);
  if (e == cudaSuccess) e = alloc(&P->off, (size_t)P->nEd + 1, s);
  if (e == cudaSuccess) e = alloc(&fill, (size_t)P->nEd + 1, s);
  if (e == cudaSuccess) e = alloc(&bsize, (size_t)P->nEd + 1, s);
  if (e == cudaSuccess) e = alloc(&P->boff, (size_t)P->nEd + 1, s);
  if (e == cudaSuccess) e = alloc(&ev, (size_t)P->nEd, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (P->nEd + 1), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(fill, 0, sizeof(int32_t) * (P->nEd + 1), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bsize, 0, sizeof(int32_t) * (P->nEd + 1), s);
  if (e == cudaSuccess && nE > 0) {
    k_patch_count<<<grid_for(nE), kThreads, 0, s>>>(m->tet, m->tface, m->tmult, nE, E.first, E.ebase, cnt, ev);
    e = launched();
  }
  if (e != cudaSuccess) { st = cuda_status(e, "ph_schwarz_create"); goto done; }
  st = exclusive_scan(cnt, P->off, P->nEd + 1, d_tot + 1, s, status);
  if (st != PH_OK) goto done;
  e = cudaMemcpyAsync(tot + 1, d_tot + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { st = cuda_status(e, "ph_schwarz_create"); goto done; }
  P->nmem = tot[1];
  e = alloc(&P->mem, (size_t)P->nmem, s);
  if (e == cudaSuccess && nE > 0) {
    k_patch_fill<<<grid_for(nE), kThreads, 0, s>>>(m->tface, m->tmult, nE, E.first, E.ebase, P->off, fill, P->mem);
    e = launched();
  }
  if (e == cudaSuccess && P->nEd > 0) {
    k_patch_sort<<<grid_for(P->nEd), kThreads, 0, s>>>(P->nEd, P->off, P->mem, bsize);
    e = launched();
  }
  if (e != cudaSuccess) { st = cuda_status(e, "ph_schwarz_create"); goto done; }
  st = exclusive_scan(bsize, P->boff, P->nEd + 1, d_tot + 2, s, status);
  if (st != PH_OK) goto done;
  e = cudaMemcpyAsync(tot + 2, d_tot + 2, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { st = cuda_status(e, "ph_schwarz_create"); goto done; }
  if (bits) { st = status_from_bits(bits); goto done; }
  if (tot[2] >= ((int64_t)1 << 31) - 1) { st = PH_ERR_OVERFLOW; goto done; }

  // blocks and face slots
  e = alloc(&P->blk, (size_t)tot[2], s);
  if (e == cudaSuccess) e = alloc(&m2f, (size_t)L, s);
  if (e == cudaSuccess) e = alloc(&P->fslot, (size_t)(3 * L), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->fslot, 0, sizeof(int32_t) * 3 * L, s);
  if (e == cudaSuccess && nF > 0) {
    k_mult_to_face<<<grid_for(nF), kThreads, 0, s>>>(m->face_mult, nF, m2f);
    e = launched();
  }
  if (e == cudaSuccess && P->nEd > 0) {
    k_patch_factor<<<grid_for(P->nEd, 128), 128, 0, s>>>(P->nEd, P->off, P->mem, P->boff, m->rowptr, m->colind,
                                                         values, P->blk, status);
    k_face_slots<<<grid_for(P->nEd), kThreads, 0, s>>>(P->nEd, P->off, P->mem, ev, m2f, m->face_vtx, P->fslot);
    e = launched(2);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { st = cuda_status(e, "ph_schwarz_create"); goto done; }
  if (bits) st = status_from_bits(bits);

done:
  release_edges(E, s);
  free_async(cnt, s);
  free_async(fill, s);
  free_async(bsize, s);
  free_async(ev, s);
  free_async(m2f, s);
  free_async(d_tot, s);
  free_async(status, s);
  if (st != PH_OK) {
    schwarz_free(P, s);
    return st;
  }
  *out = P;
  return PH_OK;
}

extern "C" ph_status ph_schwarz_destroy(ph_schwarz* P, void* stream) {
  schwarz_free(P, (cudaStream_t)stream);
  return PH_OK;
}
