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
// face's T+ tet; patch members sorted; patches grouped by size (slot-major
// within a group, in edge order); each patch block extracted from the CSR and
// inverted in FP64 by Cholesky (upper triangle stored).
// Application (schwarz_apply): one thread per patch computes y_e = block^-1 r_e
// (sums in member order) with the block in registers, then one thread per
// multiplier adds the three values of its face's three edges in a fixed order
// -- no atomics, so a solve repeats bit for bit.
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
// patch counts per group.
__global__ void k_patch_sort(int64_t nEd, const int32_t* __restrict__ off, int32_t* __restrict__ mem,
                             int32_t* __restrict__ gcnt) {
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
  if (k > kSchwarzDense) atomicAdd(&gcnt[1], k);  // its diagonal: k patches of one member
  else if (k > 0) atomicAdd(&gcnt[k], 1);
}

// Patches an edge contributes to group k (for the deterministic placement).
__global__ void k_group_indicator(int64_t nEd, const int32_t* __restrict__ off, int k, int32_t* __restrict__ ind) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nEd) return;
  const int ke = off[e + 1] - off[e];
  ind[e] = (ke == k ? 1 : 0) + (k == 1 && ke > kSchwarzDense ? ke : 0);
}

// Side of face F (face_vtx order) opposite vertex s: the face's edge (lo, hi).
__device__ __forceinline__ int face_side(const int32_t* __restrict__ face_vtx, int64_t F, int2 lh) {
  const int x = face_vtx[3 * F], y = face_vtx[3 * F + 1];
  return (x != lh.x && x != lh.y) ? 0 : (y != lh.x && y != lh.y) ? 1 : 2;
}

// Edge patches of group k into the slot-major arrays, in edge order (pos from
// a scan of k_group_indicator), and each member's y position into fslot.
__global__ void k_group_place(int64_t nEd, int k, const int32_t* __restrict__ off,
                              const int32_t* __restrict__ emem, const int32_t* __restrict__ ind,
                              const int32_t* __restrict__ pos, int64_t count, int64_t mbase,
                              const int2* __restrict__ ev, const int32_t* __restrict__ m2f,
                              const int32_t* __restrict__ face_vtx, int32_t* __restrict__ mem,
                              int32_t* __restrict__ fslot) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nEd || ind[e] == 0) return;
  const int b = off[e], ke = off[e + 1] - b;
  const int2 lh = ev[e];
  for (int i = 0; i < ke; ++i) {
    // a patch of k members: member i in slot i; a wide patch's member i: its own 1-member patch
    const int64_t at = ke == k ? mbase + (int64_t)i * count + pos[e] : mbase + pos[e] + i;
    const int l = emem[b + i];
    mem[at] = l;
    fslot[3 * (int64_t)l + face_side(face_vtx, m2f[l], lh)] = (int)at;
  }
}

__device__ __forceinline__ double csr_entry(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                                            const double* __restrict__ values, int row, int col) {
  for (int j = rowptr[row]; j < rowptr[row + 1]; ++j)
    if (colind[j] == col) return values[j];
  return 0.0;
}

// Group of patch index t (patches ordered by group).
__device__ __forceinline__ int group_of(const SchwarzGroups& g, int64_t t) {
  int k = 1;
  while (k < kSchwarzDense && t >= g.first[k + 1]) ++k;
  return k;
}

// Invert each patch block: Cholesky A = G G', then A^-1 = G^-T G^-1 (upper
// triangle stored, slot-major within the group).
__global__ void k_group_factor(SchwarzGroups g, int64_t npatch, const int32_t* __restrict__ mem,
                               const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                               const double* __restrict__ values, double* __restrict__ blk, unsigned* status) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= npatch) return;
  const int k = group_of(g, t);
  const int64_t s = t - g.first[k], n = g.count[k];
  const int32_t* mm = mem + g.mbase[k] + s;  // member i at mm[i n]
  double* out = blk + g.bbase[k] + s;        // entry q at out[q n]
  constexpr int K = kSchwarzDense;
  double a[K * K];  // lower Cholesky factor, then its inverse (row-major)
  for (int i = 0; i < k; ++i)
    for (int j = 0; j <= i; ++j) a[i * K + j] = csr_entry(rowptr, colind, values, mm[i * n], mm[j * n]);
  for (int j = 0; j < k; ++j) {
    double d = a[j * K + j];
    for (int q = 0; q < j; ++q) d -= a[j * K + q] * a[j * K + q];
    if (!(d > 0.0)) {
      ph_flag(status, PH_ERR_ARG);
      return;
    }
    const double gj = sqrt(d);
    a[j * K + j] = gj;
    for (int i = j + 1; i < k; ++i) {
      double v = a[i * K + j];
      for (int q = 0; q < j; ++q) v -= a[i * K + q] * a[j * K + q];
      a[i * K + j] = v / gj;
    }
  }
  // G^-1 in place (lower triangular), column by column
  for (int j = 0; j < k; ++j) {
    a[j * K + j] = 1.0 / a[j * K + j];
    for (int i = j + 1; i < k; ++i) {
      double v = 0.0;
      for (int q = j; q < i; ++q) v -= a[i * K + q] * a[q * K + j];
      a[i * K + j] = v / a[i * K + i];
    }
  }
  // A^-1 = G^-T G^-1: (i, j) = sum_{q >= max(i, j)} Gi[q][i] Gi[q][j]
  for (int i = 0; i < k; ++i)
    for (int j = i; j < k; ++j) {
      double v = 0.0;
      for (int q = j; q < k; ++q) v += a[q * K + i] * a[q * K + j];
      out[(int64_t)upper(i, j, k) * n] = v;
    }
}

__global__ void k_mult_to_face(const int32_t* __restrict__ face_mult, int64_t nF, int32_t* __restrict__ m2f) {
  const int64_t F = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (F < nF && face_mult[F] >= 0) m2f[face_mult[F]] = (int)F;
}

// y = block^-1 r_patch for one patch of K members (slot-major group arrays,
// stride n): the packed inverse in registers, sums in member order.
template <int K>
__device__ __forceinline__ void patch_solve(int64_t s, int64_t n, const int32_t* __restrict__ mem,
                                            const double* __restrict__ blk, const double* __restrict__ r,
                                            double* __restrict__ y) {
  constexpr int NQ = K * (K + 1) / 2;
  double m[NQ], rv[K];
#pragma unroll
  for (int q = 0; q < NQ; ++q) m[q] = __ldcs(blk + q * n + s);
#pragma unroll
  for (int j = 0; j < K; ++j) rv[j] = __ldg(r + __ldg(mem + j * n + s));
#pragma unroll
  for (int i = 0; i < K; ++i) {
    double v = 0.0;
#pragma unroll
    for (int j = 0; j < K; ++j) v = fma(m[i <= j ? upper(i, j, K) : upper(j, i, K)], rv[j], v);
    y[i * n + s] = v;
  }
}

__global__ void __launch_bounds__(256) k_schwarz_patch(SchwarzGroups g, int64_t npatch,
                                                       const int32_t* __restrict__ mem,
                                                       const double* __restrict__ blk, const double* __restrict__ r,
                                                       double* __restrict__ y) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= npatch) return;
  const int k = group_of(g, t);
  const int64_t s = t - g.first[k], n = g.count[k];
  const int32_t* mm = mem + g.mbase[k];
  const double* bb = blk + g.bbase[k];
  double* yy = y + g.mbase[k];
  switch (k) {  // uniform across a warp except at the group boundaries
    case 1: patch_solve<1>(s, n, mm, bb, r, yy); break;
    case 2: patch_solve<2>(s, n, mm, bb, r, yy); break;
    case 3: patch_solve<3>(s, n, mm, bb, r, yy); break;
    case 4: patch_solve<4>(s, n, mm, bb, r, yy); break;
    case 5: patch_solve<5>(s, n, mm, bb, r, yy); break;
    case 6: patch_solve<6>(s, n, mm, bb, r, yy); break;
    case 7: patch_solve<7>(s, n, mm, bb, r, yy); break;
    case 8: patch_solve<8>(s, n, mm, bb, r, yy); break;
    default: {  // 9..kSchwarzDense members: rare; the block read entry by entry
      double rv[kSchwarzDense];
      for (int j = 0; j < k; ++j) rv[j] = __ldg(r + __ldg(mm + j * n + s));
      for (int i = 0; i < k; ++i) {
        double v = 0.0;
        for (int j = 0; j < k; ++j) v = fma(__ldg(bb + (int64_t)(i <= j ? upper(i, j, k) : upper(j, i, k)) * n + s),
                                            rv[j], v);
        yy[i * n + s] = v;
      }
    }
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
  if (P->npatch > 0)
    k_schwarz_patch<<<ph::grid_for(P->npatch), 256, 0, s>>>(P->g, P->npatch, P->mem, P->blk, r, y);
  k_schwarz_face<<<RB, RT, 0, s>>>(P->L, P->fslot, y, r, z, part, sc, init);
  return ph::launched(P->npatch > 0 ? 2 : 1);
}

}  // namespace ph_pcg

using namespace ph;

static void schwarz_free(ph_schwarz* P, cudaStream_t s) {
  if (!P) return;
  free_async(P->mem, s);
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
  int32_t *cnt = nullptr, *off = nullptr, *fill = nullptr, *emem = nullptr, *m2f = nullptr, *gcnt = nullptr;
  int32_t *ind = nullptr, *pos = nullptr;
  int2* ev = nullptr;
  int64_t* d_tot = nullptr;  // [0] nEd, [1] incidences, [2] scan scratch
  unsigned* status = nullptr;
  int64_t tot[2] = {0, 0};
  int32_t hcnt[kSchwarzDense + 1] = {0};
  unsigned bits = 0;
  ph_status st = PH_OK;
  SchwarzGroups& g = P->g;
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

  // members of each edge patch (edge order), sorted, and the group sizes
  e = alloc(&cnt, (size_t)P->nEd + 1, s);
  if (e == cudaSuccess) e = alloc(&off, (size_t)P->nEd + 1, s);
  if (e == cudaSuccess) e = alloc(&fill, (size_t)P->nEd + 1, s);
  if (e == cudaSuccess) e = alloc(&ev, (size_t)P->nEd, s);
  if (e == cudaSuccess) e = alloc(&gcnt, (size_t)kSchwarzDense + 1, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (P->nEd + 1), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(fill, 0, sizeof(int32_t) * (P->nEd + 1), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(gcnt, 0, sizeof(int32_t) * (kSchwarzDense + 1), s);
  if (e == cudaSuccess && nE > 0) {
    k_patch_count<<<grid_for(nE), kThreads, 0, s>>>(m->tet, m->tface, m->tmult, nE, E.first, E.ebase, cnt, ev);
    e = launched();
  }
  if (e != cudaSuccess) { st = cuda_status(e, "ph_schwarz_create"); goto done; }
  st = exclusive_scan(cnt, off, P->nEd + 1, d_tot + 1, s, status);
  if (st != PH_OK) goto done;
  e = cudaMemcpyAsync(tot + 1, d_tot + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { st = cuda_status(e, "ph_schwarz_create"); goto done; }
  P->nmem = tot[1];
  e = alloc(&emem, (size_t)P->nmem, s);
  if (e == cudaSuccess && nE > 0) {
    k_patch_fill<<<grid_for(nE), kThreads, 0, s>>>(m->tface, m->tmult, nE, E.first, E.ebase, off, fill, emem);
    e = launched();
  }
  if (e == cudaSuccess && P->nEd > 0) {
    k_patch_sort<<<grid_for(P->nEd), kThreads, 0, s>>>(P->nEd, off, emem, gcnt);
    e = launched();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(hcnt, gcnt, sizeof hcnt, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { st = cuda_status(e, "ph_schwarz_create"); goto done; }
  if (bits) { st = status_from_bits(bits); goto done; }

  // group table: patches ordered by size, slot-major arrays per group
  g.first[1] = 0;
  for (int k = 1; k <= kSchwarzDense; ++k) {
    g.count[k] = hcnt[k];
    g.first[k + 1] = g.first[k] + g.count[k];
    g.mbase[k] = k == 1 ? 0 : g.mbase[k - 1] + (int64_t)(k - 1) * g.count[k - 1];
    g.bbase[k] = k == 1 ? 0 : g.bbase[k - 1] + (int64_t)(k - 1) * k / 2 * g.count[k - 1];
  }
  P->npatch = g.first[kSchwarzDense + 1];
  P->nblk = g.bbase[kSchwarzDense] + (int64_t)kSchwarzDense * (kSchwarzDense + 1) / 2 * g.count[kSchwarzDense];
  if (P->nblk >= ((int64_t)1 << 31) - 1) { st = PH_ERR_OVERFLOW; goto done; }

  // placement (one deterministic pass per occupied group) and face slots
  e = alloc(&P->mem, (size_t)P->nmem, s);
  if (e == cudaSuccess) e = alloc(&P->blk, (size_t)P->nblk, s);
  if (e == cudaSuccess) e = alloc(&m2f, (size_t)L, s);
  if (e == cudaSuccess) e = alloc(&P->fslot, (size_t)(3 * L), s);
  if (e == cudaSuccess) e = alloc(&ind, (size_t)P->nEd + 1, s);
  if (e == cudaSuccess) e = alloc(&pos, (size_t)P->nEd + 1, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->fslot, 0, sizeof(int32_t) * 3 * L, s);
  if (e == cudaSuccess && nF > 0) {
    k_mult_to_face<<<grid_for(nF), kThreads, 0, s>>>(m->face_mult, nF, m2f);
    e = launched();
  }
  if (e != cudaSuccess) { st = cuda_status(e, "ph_schwarz_create"); goto done; }
  for (int k = 1; k <= kSchwarzDense && P->nEd > 0; ++k) {
    if (g.count[k] == 0) continue;
    k_group_indicator<<<grid_for(P->nEd), kThreads, 0, s>>>(P->nEd, off, k, ind);
    e = launched();
    if (e == cudaSuccess) e = cudaMemsetAsync(ind + P->nEd, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) { st = cuda_status(e, "ph_schwarz_create"); goto done; }
    st = exclusive_scan(ind, pos, P->nEd + 1, d_tot + 2, s, status);
    if (st != PH_OK) goto done;
    k_group_place<<<grid_for(P->nEd), kThreads, 0, s>>>(P->nEd, k, off, emem, ind, pos, g.count[k], g.mbase[k], ev,
                                                        m2f, m->face_vtx, P->mem, P->fslot);
    e = launched();
    if (e != cudaSuccess) { st = cuda_status(e, "ph_schwarz_create"); goto done; }
  }
  if (P->npatch > 0) {
    k_group_factor<<<grid_for(P->npatch, 128), 128, 0, s>>>(g, P->npatch, P->mem, m->rowptr, m->colind, values,
                                                            P->blk, status);
    e = launched();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { st = cuda_status(e, "ph_schwarz_create"); goto done; }
  if (bits) st = status_from_bits(bits);

done:
  release_edges(E, s);
  for (void* q : {(void*)cnt, (void*)off, (void*)fill, (void*)emem, (void*)m2f, (void*)gcnt, (void*)ind, (void*)pos,
                  (void*)ev, (void*)d_tot, (void*)status})
    free_async(q, s);
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
