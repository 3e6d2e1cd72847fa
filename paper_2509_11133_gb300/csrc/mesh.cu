// Mesh construction on the device: face-to-tetrahedron connectivity
// (Section 3.3), face / multiplier numbering, the CSR pattern of the condensed
// face system and per-element geometry.
//
// Connectivity.  The paper builds faces from edge-to-tet sparse maps
// (Listings EdgeNum2Tetra, FacesUp).  Here every local face becomes a key
// (v0 < v1 < v2) that is counting-sorted into buckets by its largest vertex v2
// (histogram, scan, scatter; mesh order keeps the scatter local; on refined
// meshes the largest vertex spreads keys more evenly than the smallest), and
// the keys of a bucket are matched against each other.  The result is the
// paper's numbering: a face's id is the rank of its first occurrence in
// (tet, local face) order and the tet of that occurrence is T+; it does not
// depend on the order of entries inside a bucket.
#include <math.h>
#include <string.h>

#include <mutex>

#include "ph_internal.cuh"

namespace {

__device__ __forceinline__ int comp(int4 v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }

// Local face k of T = [a b c d]: [a b c], [a c d], [a d b], [d c b] (Section 2.2).
__device__ __forceinline__ int3 local_face(int4 v, int k) {
  switch (k) {
    case 0: return make_int3(v.x, v.y, v.z);
    case 1: return make_int3(v.x, v.z, v.w);
    case 2: return make_int3(v.x, v.w, v.y);
    default: return make_int3(v.w, v.z, v.y);
  }
}

__device__ __forceinline__ int3 sort3(int3 a) {
  int x = a.x, y = a.y, z = a.z, t;
  if (y < x) { t = x; x = y; y = t; }
  if (z < y) { t = y; y = z; z = t; }
  if (y < x) { t = x; x = y; y = t; }
  return make_int3(x, y, z);
}

__device__ __forceinline__ bool valid_tet(int4 v, int64_t nC) {
  bool in = v.x >= 0 && v.y >= 0 && v.z >= 0 && v.w >= 0 && v.x < nC && v.y < nC && v.z < nC && v.w < nC;
  bool distinct = v.x != v.y && v.x != v.z && v.x != v.w && v.y != v.z && v.y != v.w && v.z != v.w;
  return in && distinct;
}

__device__ __forceinline__ bool valid_tri(int3 v, int64_t nC) {
  bool in = v.x >= 0 && v.y >= 0 && v.z >= 0 && v.x < nC && v.y < nC && v.z < nC;
  return in && v.x != v.y && v.x != v.z && v.y != v.z;
}

__device__ __forceinline__ int3 neumann_tri(const int32_t* nb, int64_t i) {
  return make_int3(nb[3 * i], nb[3 * i + 1], nb[3 * i + 2]);
}

// 1. histogram of face keys by largest vertex
__global__ void k_face_count(const int4* __restrict__ tet, int64_t nE, int64_t nC, const int32_t* __restrict__ nb,
                             int64_t nN, int32_t* __restrict__ cnt, unsigned* status) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < nE) {
    int4 v = tet[i];
    if (!valid_tet(v, nC)) { ph_flag(status, PH_ERR_ARG); return; }
#pragma unroll
    for (int k = 0; k < 4; ++k) atomicAdd(&cnt[sort3(local_face(v, k)).z], 1);
  } else if (i < nE + nN) {
    int3 f = neumann_tri(nb, i - nE);
    if (!valid_tri(f, nC)) { ph_flag(status, PH_ERR_ARG); return; }
    atomicAdd(&cnt[sort3(f).z], 1);
  }
}

// 2. scatter keys into buckets (all keys of a bucket share v2): entry =
//    (v0, v1, v2, slot), slot = 4t+k for tet faces and 4nE+i for Neumann
//    triples.  cnt counts down to 0.
__global__ void k_face_fill(const int4* __restrict__ tet, int64_t nE, int64_t nC, const int32_t* __restrict__ nb,
                            int64_t nN, const int32_t* __restrict__ start, int32_t* __restrict__ cnt,
                            int4* __restrict__ entries) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < nE) {
    int4 v = tet[i];
    if (!valid_tet(v, nC)) return;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      int3 s = sort3(local_face(v, k));
      int pos = start[s.z] + atomicSub(&cnt[s.z], 1) - 1;
      entries[pos] = make_int4(s.x, s.y, s.z, (int)(4 * i + k));
    }
  } else if (i < nE + nN) {
    int3 f = neumann_tri(nb, i - nE);
    if (!valid_tri(f, nC)) return;
    int3 s = sort3(f);
    int pos = start[s.z] + atomicSub(&cnt[s.z], 1) - 1;
    entries[pos] = make_int4(s.x, s.y, s.z, (int)i + 3 * (int)nE);  // slot 4nE + (i - nE)
  }
}

// Scan entries[j0, j1) for (v0, v1) == (e.x, e.y) (v2 is the bucket's);
// counts tet and Neumann matches.  Four independent loads per step.
__device__ __forceinline__ void scan_bucket(const int4* __restrict__ entries, int j0, int j1, int skip, int4 e,
                                            int64_t ntet, int& nt, int& nn, int& tm) {
  int j = j0;
  for (; j + 3 < j1; j += 4) {
    const int4 k0 = entries[j], k1 = entries[j + 1], k2 = entries[j + 2], k3 = entries[j + 3];
    const int4 kk[4] = {k0, k1, k2, k3};
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (kk[u].x == e.x && kk[u].y == e.y && j + u != skip) {
        if (kk[u].w < ntet) { ++nt; tm = kk[u].w; } else { ++nn; }
      }
  }
  for (; j < j1; ++j) {
    const int4 k = entries[j];
    if (k.x == e.x && k.y == e.y && j != skip) {
      if (k.w < ntet) { ++nt; tm = k.w; } else { ++nn; }
    }
  }
}

// 3. match equal keys inside a bucket (all keys of a bucket share v2).
//    mate[slot] of a tet slot: the other tet slot of the face, -1 (Dirichlet
//    boundary, the initial value) or -2 (Neumann boundary).  A tet entry
//    compares itself with the LATER entries of its bucket only and writes both
//    mates of a pair, so each pair is found once; a second match marks a face
//    in three tets (or a Neumann triple on an interior face).  Neumann entries
//    (boundary only, few) scan the whole bucket and must match exactly one tet
//    entry.
__global__ void k_face_match(const int4* __restrict__ entries, int64_t nent, const int32_t* __restrict__ start,
                             int64_t nE, int32_t* __restrict__ mate, unsigned* status) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nent) return;
  const int4 e = entries[i];
  const int hi = start[e.z + 1];
  const int64_t ntet = 4 * nE;
  int nt = 0, nn = 0, tm = -1;
  if (e.w < ntet) {
    scan_bucket(entries, (int)i + 1, hi, -1, e, ntet, nt, nn, tm);
    if (nt + nn >= 2) ph_flag(status, nn > 0 ? PH_ERR_ARG : PH_ERR_NONMANIFOLD);
    if (nt == 1) {
      mate[e.w] = tm;
      mate[tm] = e.w;
    } else if (nn == 1) {
      mate[e.w] = -2;
    }
  } else {
    scan_bucket(entries, start[e.z], hi, (int)i, e, ntet, nt, nn, tm);
    if (nt != 1 || nn != 0) ph_flag(status, PH_ERR_ARG);
    else mate[tm] = -2;
  }
}

__device__ __forceinline__ bool is_first(int m, int s) { return m < 0 || m > s; }

// 4. number of faces whose first occurrence is in tet t
__global__ void k_new_count(const int4* __restrict__ mate4, int64_t nE, int32_t* __restrict__ newc) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nE) return;
  int4 m = mate4[t];
  int s = (int)(4 * t);
  newc[t] = is_first(m.x, s) + is_first(m.y, s + 1) + is_first(m.z, s + 2) + is_first(m.w, s + 3);
}

__device__ __forceinline__ int first_rank(int4 m, int s0, int k) {
  int r = 0;
  if (k > 0) r += is_first(m.x, s0);
  if (k > 1) r += is_first(m.y, s0 + 1);
  if (k > 2) r += is_first(m.z, s0 + 2);
  return r;
}

// 5. per tet: face ids, T+/T-, T+'s tuple, kind and non-Neumann flag of the
//    faces it owns (first occurrences).
__global__ void k_face_emit(const int4* __restrict__ tet, int64_t nE, const int4* __restrict__ mate4,
                            const int32_t* __restrict__ fbase, int4* __restrict__ tface, int2* __restrict__ face_tet,
                            int32_t* __restrict__ face_vtx, int8_t* __restrict__ face_kind,
                            int32_t* __restrict__ flag) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nE) return;
  int4 v = tet[t];
  int4 m = mate4[t];
  int s0 = (int)(4 * t);
  int out[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    int mk = comp(m, k);
    if (is_first(mk, s0 + k)) {
      int F = fbase[t] + first_rank(m, s0, k);
      out[k] = F;
      face_tet[F] = make_int2((int)t, mk >= 0 ? (mk >> 2) : -1);
      int3 lf = local_face(v, k);
      face_vtx[3 * (int64_t)F] = lf.x;
      face_vtx[3 * (int64_t)F + 1] = lf.y;
      face_vtx[3 * (int64_t)F + 2] = lf.z;
      const int kind = mk >= 0 ? 0 : (mk == -1 ? 1 : 2);
      face_kind[F] = (int8_t)kind;
      flag[F] = kind != 2;
    } else {
      int t2 = mk >> 2, k2 = mk & 3;
      int F = fbase[t2] + first_rank(mate4[t2], 4 * t2, k2);
      out[k] = (int)((unsigned)F | 0x80000000u);
    }
  }
  tface[t] = make_int4(out[0], out[1], out[2], out[3]);
}

// Element geometry (needs only the inputs, so it runs beside connectivity):
// E = rows P_i - P_0 (i = 1..3), G_e = E E', GT = G_e T0^-1 = G_e - (G_e 1) 1'/4
// (T0 = I + 1 1'), |det E|, 1/|det E|.
__global__ void k_tet_geom(const double* __restrict__ coord, const int4* __restrict__ tet, int64_t nE,
                           double* __restrict__ geo, unsigned* status) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nE) return;
  const int4 v = tet[t];
  const double* p0 = coord + 3 * (int64_t)v.x;
  const double* p1 = coord + 3 * (int64_t)v.y;
  const double* p2 = coord + 3 * (int64_t)v.z;
  const double* p3 = coord + 3 * (int64_t)v.w;
  const double e1x = p1[0] - p0[0], e1y = p1[1] - p0[1], e1z = p1[2] - p0[2];
  const double e2x = p2[0] - p0[0], e2y = p2[1] - p0[1], e2z = p2[2] - p0[2];
  const double e3x = p3[0] - p0[0], e3y = p3[1] - p0[1], e3z = p3[2] - p0[2];
  const double det = e1x * (e2y * e3z - e2z * e3y) + e1y * (e2z * e3x - e2x * e3z) + e1z * (e2x * e3y - e2y * e3x);
  const double adet = ph::neg_if(det, __double2hiint(det) < 0);  // |det| on the sign bit
  if (!ph::pos_finite(adet)) ph_flag(status, PH_ERR_DEGENERATE);
  const double g00 = e1x * e1x + e1y * e1y + e1z * e1z, g01 = e1x * e2x + e1y * e2y + e1z * e2z;
  const double g02 = e1x * e3x + e1y * e3y + e1z * e3z, g11 = e2x * e2x + e2y * e2y + e2z * e2z;
  const double g12 = e2x * e3x + e2y * e3y + e2z * e3z, g22 = e3x * e3x + e3y * e3y + e3z * e3z;
  const double r0 = 0.25 * (g00 + g01 + g02), r1 = 0.25 * (g01 + g11 + g12), r2 = 0.25 * (g02 + g12 + g22);
  double2* gg = reinterpret_cast<double2*>(geo + PH_GEO_STRIDE * t);
  gg[0] = make_double2(g00, g01);
  gg[1] = make_double2(g02, g11);
  gg[2] = make_double2(g12, g22);
  gg[3] = make_double2(g00 - r0, g01 - r0);
  gg[4] = make_double2(g02 - r0, g01 - r1);
  gg[5] = make_double2(g11 - r1, g12 - r1);
  gg[6] = make_double2(g02 - r2, g12 - r2);
  gg[7] = make_double2(g22 - r2, adet);
  gg[8] = make_double2(ph::rcp_newton(adet), 0.0);
}

// 6. face areas 1/2 |(P_z - P_x) x (P_y - P_x)| (one thread per face)
__global__ void k_face_area(const double* __restrict__ coord, const int32_t* __restrict__ face_vtx, int64_t nF,
                            double* __restrict__ area) {
  int64_t F = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (F >= nF) return;
  const double* x = coord + 3 * (int64_t)face_vtx[3 * F];
  const double* y = coord + 3 * (int64_t)face_vtx[3 * F + 1];
  const double* z = coord + 3 * (int64_t)face_vtx[3 * F + 2];
  double u0 = z[0] - x[0], u1 = z[1] - x[1], u2 = z[2] - x[2];
  double v0 = y[0] - x[0], v1 = y[1] - x[1], v2 = y[2] - x[2];
  double cx = u1 * v2 - u2 * v1, cy = u2 * v0 - u0 * v2, cz = u0 * v1 - u1 * v0;
  area[F] = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
}

__global__ void k_mult_fix(int32_t* __restrict__ face_mult, const int8_t* __restrict__ face_kind, int64_t nF) {
  int64_t F = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (F < nF && face_kind[F] == 2) face_mult[F] = -1;
}

// 7. per-slot multiplier ids and row lengths: row l(F) = 1 + sum over F's
//    tets of (non-Neumann faces of the tet) - 1.
__global__ void k_tet_mult(const int4* __restrict__ tface, int64_t nE, const int32_t* __restrict__ face_mult,
                           const int2* __restrict__ face_tet, int4* __restrict__ tmult, int32_t* __restrict__ rowlen) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nE) return;
  int4 tf = tface[t];
  int l[4], o[4];
  int mT = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    int F = comp(tf, k) & PH_ID_MASK;
    l[k] = face_mult[F];
    mT += l[k] >= 0;
    bool bnd = face_tet[F].y < 0;
    o[k] = l[k] < 0 ? PH_NO_MULT : (int)((unsigned)l[k] | (bnd ? PH_BND_BIT : 0u));
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (l[k] >= 0) atomicAdd(&rowlen[l[k]], mT - 1 + (comp(tf, k) >= 0 ? 1 : 0));
  tmult[t] = make_int4(o[0], o[1], o[2], o[3]);
}

// 8. column indices of each row (ascending), the diagonal position, and each
//    slot's scatter positions: tpos = diagonal, trel = rank offsets of the
//    other three local faces (4-bit two's complement, m != k ascending).
__global__ void k_row_fill(const int2* __restrict__ face_tet, const int4* __restrict__ tface,
                           const int4* __restrict__ tmult, const int32_t* __restrict__ face_mult, int64_t nF,
                           const int32_t* __restrict__ rowptr, int32_t* __restrict__ colind,
                           int32_t* __restrict__ rowdiag, int32_t* __restrict__ tpos,
                           unsigned short* __restrict__ trel, unsigned* status) {
  int64_t F = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (F >= nF) return;
  int l = face_mult[F];
  if (l < 0) return;
  int2 ft = face_tet[F];
  int cols[7];
  int n = 0;
  cols[n++] = l;
  int tts[2] = {ft.x, ft.y};
  for (int side = 0; side < 2; ++side) {
    int T = tts[side];
    if (T < 0) continue;
    int4 tf = tface[T], tm = tmult[T];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int G = comp(tf, j) & PH_ID_MASK;
      int mj = comp(tm, j);
      if (G != F && mj != PH_NO_MULT && n < 7) cols[n++] = mj & PH_ID_MASK;
    }
  }
  for (int i = 1; i < n; ++i) {  // insertion sort of <= 7 ids
    int x = cols[i], j = i - 1;
    while (j >= 0 && cols[j] > x) { cols[j + 1] = cols[j]; --j; }
    cols[j + 1] = x;
  }
  int base = rowptr[l];
  if (rowptr[l + 1] - base != n) { ph_flag(status, PH_ERR_ARG); return; }
  int rl = 0;
  for (int i = 0; i < n; ++i) {
    colind[base + i] = cols[i];
    if (cols[i] == l) rl = i;
  }
  rowdiag[l] = base + rl;
  for (int side = 0; side < 2; ++side) {
    int T = tts[side];
    if (T < 0) continue;
    int4 tf = tface[T], tm = tmult[T];
    int k = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if ((comp(tf, j) & PH_ID_MASK) == F) k = j;
    unsigned bits = 0;
    int idx = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      if (m == k) continue;
      int mm = comp(tm, m);
      if (mm != PH_NO_MULT) {
        int lm = mm & PH_ID_MASK, r = 0;
        for (int i = 0; i < n; ++i)
          if (cols[i] == lm) r = i;
        bits |= ((unsigned)(r - rl) & 0xFu) << (4 * idx);
      }
      ++idx;
    }
    tpos[4 * (int64_t)T + k] = base + rl;
    trel[4 * (int64_t)T + k] = (unsigned short)bits;
  }
}

__global__ void k_face_centroid(const double* __restrict__ coord, const int32_t* __restrict__ face_vtx, int64_t nF,
                                double* __restrict__ out) {
  int64_t F = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (F >= nF) return;
  const double* x = coord + 3 * (int64_t)face_vtx[3 * F];
  const double* y = coord + 3 * (int64_t)face_vtx[3 * F + 1];
  const double* z = coord + 3 * (int64_t)face_vtx[3 * F + 2];
#pragma unroll
  for (int d = 0; d < 3; ++d) out[3 * F + d] = (x[d] + y[d] + z[d]) / 3.0;
}

struct Counters {
  int64_t total;
  unsigned status;
  unsigned pad;
};

}  // namespace

using namespace ph;

static void mesh_free(ph_mesh* m, cudaStream_t s) {
  if (!m) return;
  void* ptrs[] = {m->coord, m->tet, m->tface, m->tmult, m->tpos, m->trel, m->geo, m->face_tet, m->face_vtx,
                  m->face_kind, m->face_mult, m->face_area, m->rowptr, m->colind, m->rowdiag, m->status};
  for (void* p : ptrs) free_async(p, s);
  delete m;
}

// Synchronise and read n device int64 counters and the status word.
static ph_status read_counters(const int64_t* d_tot, int n, unsigned* d_status, cudaStream_t s, int64_t* tot,
                               unsigned* status) {
  cudaError_t e = cudaMemcpyAsync(tot, d_tot, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(status, d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return cuda_status(e, "mesh_create sync");
}

// Two internal streams per device for ph_mesh_create: connectivity (integer
// and memory work) runs on a high-priority stream and element geometry (FP64
// work) on a low-priority one, so geometry blocks fill the SM slots the
// connectivity kernels leave free.  Both are forked from and joined back into
// the caller's stream.
static std::mutex g_aux_mu;
static cudaStream_t g_hi[64], g_lo[64];

static cudaError_t aux_streams(int dev, cudaStream_t* hi, cudaStream_t* lo) {
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_aux_mu);
  if (!g_hi[dev]) {
    int least = 0, greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e != cudaSuccess) return e;
    e = cudaStreamCreateWithPriority(&g_hi[dev], cudaStreamNonBlocking, greatest);
    if (e != cudaSuccess) return e;
    e = cudaStreamCreateWithPriority(&g_lo[dev], cudaStreamNonBlocking, least);
    if (e != cudaSuccess) return e;
  }
  *hi = g_hi[dev];
  *lo = g_lo[dev];
  return cudaSuccess;
}

#define PH_TRY(expr)                    \
  do {                                  \
    st = (expr);                        \
    if (st != PH_OK) goto fail;         \
  } while (0)
#define PH_CU(expr, what) PH_TRY(cuda_status((expr), what))

extern "C" ph_status ph_mesh_create(const double* coord, int64_t nC, const int32_t* tet, int64_t nE,
                                    const int32_t* neumann, int64_t nN, void* stream, ph_mesh** out) {
  if (!out) return PH_ERR_ARG;
  *out = nullptr;
  if (nE < 0 || nC < 0 || nN < 0 || (nE > 0 && (!coord || !tet)) || (nN > 0 && !neumann)) return PH_ERR_ARG;
  if (4 * nE + nN >= ((int64_t)1 << 31) - 1 || nC >= ((int64_t)1 << 31) - 1) return PH_ERR_OVERFLOW;
  cudaStream_t us = (cudaStream_t)stream;  // caller's stream: fork and join only
  cudaStream_t s = nullptr, g = nullptr;    // connectivity (high priority), geometry (low)
  cudaEvent_t ev_in = nullptr, ev_emit = nullptr, ev_geo = nullptr, ev_done = nullptr;
  bool forked = false;
  ph_status st = PH_OK;
  ph_mesh* m = new ph_mesh();
  memset(m, 0, sizeof *m);
  int32_t *cnt = nullptr, *start = nullptr, *mate = nullptr, *newc = nullptr, *flag = nullptr, *rowlen = nullptr;
  int4* entries = nullptr;
  int64_t* d_tot = nullptr;  // [0] scan total, [1] L, [2] nnz
  int64_t tot[3] = {0, 0, 0};
  unsigned bits = 0;
  const int64_t nent = 4 * nE + nN;
  PH_CU(cudaGetDevice(&m->device), "cudaGetDevice");
  PH_CU(aux_streams(m->device, &s, &g), "internal streams");
  PH_CU(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming), "event");
  PH_CU(cudaEventCreateWithFlags(&ev_emit, cudaEventDisableTiming), "event");
  PH_CU(cudaEventCreateWithFlags(&ev_geo, cudaEventDisableTiming), "event");
  PH_CU(cudaEventCreateWithFlags(&ev_done, cudaEventDisableTiming), "event");
  // the inputs are ordered on the caller's stream
  PH_CU(cudaEventRecord(ev_in, us), "event");
  PH_CU(cudaStreamWaitEvent(s, ev_in, 0), "event");
  forked = true;
  m->nE = nE;
  m->nC = nC;
  PH_CU(alloc(&m->status, 1, s), "alloc");
  PH_CU(cudaMemsetAsync(m->status, 0, sizeof(unsigned), s), "memset");
  PH_CU(alloc(&d_tot, 3, s), "alloc");
  PH_CU(alloc(&m->coord, (size_t)(3 * nC), s), "alloc coord");
  PH_CU(alloc(&m->tet, (size_t)nE, s), "alloc tet");
  PH_CU(alloc(&m->geo, (size_t)(PH_GEO_STRIDE * nE), s), "alloc");
  if (nC > 0) PH_CU(cudaMemcpyAsync(m->coord, coord, sizeof(double) * 3 * nC, cudaMemcpyDeviceToDevice, s), "copy");
  if (nE > 0) PH_CU(cudaMemcpyAsync(m->tet, tet, sizeof(int4) * nE, cudaMemcpyDeviceToDevice, s), "copy");

  // --- element geometry on the low-priority stream ---------------------------
  PH_CU(cudaEventRecord(ev_in, s), "event");
  PH_CU(cudaStreamWaitEvent(g, ev_in, 0), "event");
  if (nE > 0) {
    k_tet_geom<<<grid_for(nE), kThreads, 0, g>>>(m->coord, m->tet, nE, m->geo, m->status);
    PH_CU(launched(), "k_tet_geom");
  }

  // --- connectivity -------------------------------------------------------
  PH_CU(alloc(&cnt, (size_t)nC + 1, s), "alloc");
  PH_CU(alloc(&start, (size_t)nC + 1, s), "alloc");
  PH_CU(alloc(&entries, (size_t)nent, s), "alloc");
  PH_CU(alloc(&mate, (size_t)(4 * nE), s), "alloc");
  PH_CU(alloc(&newc, (size_t)nE + 1, s), "alloc");
  PH_CU(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * ((size_t)nC + 1), s), "memset");
  PH_CU(cudaMemsetAsync(mate, 0xFF, sizeof(int32_t) * 4 * nE, s), "memset");
  if (nent > 0) {
    k_face_count<<<grid_for(nE + nN), kThreads, 0, s>>>(m->tet, nE, nC, neumann, nN, cnt, m->status);
    PH_CU(launched(), "k_face_count");
  }
  PH_TRY(exclusive_scan(cnt, start, nC + 1, d_tot, s));
  if (nent > 0) {
    k_face_fill<<<grid_for(nE + nN), kThreads, 0, s>>>(m->tet, nE, nC, neumann, nN, start, cnt, entries);
    PH_CU(launched(), "k_face_fill");
    k_face_match<<<grid_for(nent), kThreads, 0, s>>>(entries, nent, start, nE, mate, m->status);
    PH_CU(launched(), "k_face_match");
  }
  if (nE > 0) {
    k_new_count<<<grid_for(nE), kThreads, 0, s>>>(reinterpret_cast<int4*>(mate), nE, newc);
    PH_CU(launched(), "k_new_count");
  }
  PH_CU(cudaMemsetAsync(newc + nE, 0, sizeof(int32_t), s), "memset");
  PH_TRY(exclusive_scan(newc, newc, nE + 1, d_tot, s));
  PH_TRY(read_counters(d_tot, 1, m->status, s, tot, &bits));
  if (bits) { st = status_from_bits(bits); goto fail; }
  if (tot[0] >= ((int64_t)1 << 31) - 1) { st = PH_ERR_OVERFLOW; goto fail; }
  m->nF = tot[0];
  free_async(cnt, s); cnt = nullptr;
  free_async(start, s); start = nullptr;
  free_async(entries, s); entries = nullptr;

  PH_CU(alloc(&m->tface, (size_t)nE, s), "alloc");
  PH_CU(alloc(&m->face_tet, (size_t)m->nF, s), "alloc");
  PH_CU(alloc(&m->face_vtx, (size_t)(3 * m->nF), s), "alloc");
  PH_CU(alloc(&m->face_kind, (size_t)m->nF, s), "alloc");
  PH_CU(alloc(&m->face_mult, (size_t)m->nF + 1, s), "alloc");
  PH_CU(alloc(&m->face_area, (size_t)m->nF, s), "alloc");
  PH_CU(alloc(&flag, (size_t)m->nF + 1, s), "alloc");
  if (nE > 0) {
    k_face_emit<<<grid_for(nE), kThreads, 0, s>>>(m->tet, nE, reinterpret_cast<int4*>(mate), newc, m->tface,
                                                  m->face_tet, m->face_vtx, m->face_kind, flag);
    PH_CU(launched(), "k_face_emit");
  }
  free_async(mate, s); mate = nullptr;
  free_async(newc, s); newc = nullptr;
  // face areas on the second stream (after the face tuples exist)
  PH_CU(cudaEventRecord(ev_emit, s), "event");
  PH_CU(cudaStreamWaitEvent(g, ev_emit, 0), "event");
  if (m->nF > 0) {
    k_face_area<<<grid_for(m->nF), kThreads, 0, g>>>(m->coord, m->face_vtx, m->nF, m->face_area);
    PH_CU(launched(), "k_face_area");
  }

  // --- multipliers and CSR pattern ----------------------------------------
  PH_CU(cudaMemsetAsync(flag + m->nF, 0, sizeof(int32_t), s), "memset");
  PH_TRY(exclusive_scan(flag, m->face_mult, m->nF + 1, d_tot + 1, s));  // L -> d_tot[1]
  if (m->nF > 0) {
    k_mult_fix<<<grid_for(m->nF), kThreads, 0, s>>>(m->face_mult, m->face_kind, m->nF);
    PH_CU(launched(), "k_mult_fix");
  }
  free_async(flag, s); flag = nullptr;
  // rows are indexed by multiplier id < L <= nF: size the row arrays by nF
  // (rows L..nF-1 stay empty) and learn L with nnz at the next synchronisation
  PH_CU(alloc(&m->tmult, (size_t)nE, s), "alloc");
  PH_CU(alloc(&rowlen, (size_t)m->nF + 1, s), "alloc");
  PH_CU(alloc(&m->rowptr, (size_t)m->nF + 1, s), "alloc");
  PH_CU(cudaMemsetAsync(rowlen, 0, sizeof(int32_t) * (m->nF + 1), s), "memset");
  if (nE > 0) {
    k_tet_mult<<<grid_for(nE), kThreads, 0, s>>>(m->tface, nE, m->face_mult, m->face_tet, m->tmult, rowlen);
    PH_CU(launched(), "k_tet_mult");
  }
  PH_TRY(exclusive_scan(rowlen, m->rowptr, m->nF + 1, d_tot + 2, s));  // nnz -> d_tot[2]
  free_async(rowlen, s); rowlen = nullptr;
  PH_TRY(read_counters(d_tot, 3, m->status, s, tot, &bits));
  if (bits) { st = status_from_bits(bits); goto fail; }
  if (tot[2] >= ((int64_t)1 << 31) - 1) { st = PH_ERR_OVERFLOW; goto fail; }
  m->L = tot[1];
  m->nnz = tot[2];

  // --- CSR columns and scatter positions ----------------------------------
  PH_CU(alloc(&m->colind, (size_t)m->nnz, s), "alloc");
  PH_CU(alloc(&m->rowdiag, (size_t)m->L, s), "alloc");
  PH_CU(alloc(&m->tpos, (size_t)nE, s), "alloc");
  PH_CU(alloc(&m->trel, (size_t)nE, s), "alloc");
  PH_CU(cudaMemsetAsync(m->tpos, 0, sizeof(int4) * nE, s), "memset");
  PH_CU(cudaMemsetAsync(m->trel, 0, sizeof(ushort4) * nE, s), "memset");
  if (m->nF > 0) {
    k_row_fill<<<grid_for(m->nF), kThreads, 0, s>>>(m->face_tet, m->tface, m->tmult, m->face_mult, m->nF, m->rowptr,
                                                    m->colind, m->rowdiag, reinterpret_cast<int32_t*>(m->tpos),
                                                    reinterpret_cast<unsigned short*>(m->trel), m->status);
    PH_CU(launched(), "k_row_fill");
  }
  // join the geometry stream, then report any error of either stream
  PH_CU(cudaEventRecord(ev_geo, g), "event");
  PH_CU(cudaStreamWaitEvent(s, ev_geo, 0), "event");
  free_async(d_tot, s); d_tot = nullptr;
  {
    unsigned b2 = 0;
    PH_CU(cudaMemcpyAsync(&b2, m->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "copy");
    PH_CU(cudaStreamSynchronize(s), "sync");
    if (b2) { st = status_from_bits(b2); goto fail; }
  }
  // later work on the caller's stream sees the finished mesh
  PH_CU(cudaEventRecord(ev_done, s), "event");
  PH_CU(cudaStreamWaitEvent(us, ev_done, 0), "event");
  forked = false;
  // face kinds: every interior face has two slots and a boundary face one,
  // so 4 nE = 2 nFi + (nF - nFi); Neumann faces are the ones without multiplier
  m->nFi = 4 * nE - m->nF;
  m->nFn = m->nF - m->L;
  m->nFd = m->nF - m->nFi - m->nFn;
  cudaEventDestroy(ev_in);
  cudaEventDestroy(ev_emit);
  cudaEventDestroy(ev_geo);
  cudaEventDestroy(ev_done);
  *out = m;
  return PH_OK;

fail:
  if (forked && g && s && ev_geo) {  // nothing is freed before the geometry stream is done
    cudaEventRecord(ev_geo, g);
    cudaStreamWaitEvent(s, ev_geo, 0);
  }
  if (!s) s = us;
  free_async(cnt, s);
  free_async(start, s);
  free_async(entries, s);
  free_async(mate, s);
  free_async(newc, s);
  free_async(flag, s);
  free_async(rowlen, s);
  free_async(d_tot, s);
  mesh_free(m, s);
  if (ev_in) cudaEventDestroy(ev_in);
  if (ev_emit) cudaEventDestroy(ev_emit);
  if (forked && ev_done) {  // the caller's stream waits for the frees
    cudaEventRecord(ev_done, s);
    cudaStreamWaitEvent(us, ev_done, 0);
  }
  if (ev_geo) cudaEventDestroy(ev_geo);
  if (ev_done) cudaEventDestroy(ev_done);
  return st;
}

extern "C" ph_status ph_mesh_destroy(ph_mesh* mesh, void* stream) {
  if (!mesh) return PH_OK;
  mesh_free(mesh, (cudaStream_t)stream);
  return PH_OK;
}

extern "C" ph_status ph_mesh_info(const ph_mesh* m, ph_info* out) {
  if (!m || !out) return PH_ERR_ARG;
  out->nE = m->nE;
  out->nC = m->nC;
  out->nF = m->nF;
  out->nF_interior = m->nFi;
  out->nF_dirichlet = m->nFd;
  out->nF_neumann = m->nFn;
  out->L = m->L;
  out->nnz = m->nnz;
  return PH_OK;
}

extern "C" ph_status ph_mesh_faces(const ph_mesh* m, int32_t* tet_face, int32_t* face_tet, int32_t* face_vtx,
                                   int8_t* face_kind, int32_t* face_mult, double* face_centroid, double* face_area,
                                   void* stream) {
  if (!m) return PH_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  const int64_t nE = m->nE, nF = m->nF;
  if (tet_face && nE) e = cudaMemcpyAsync(tet_face, m->tface, sizeof(int4) * nE, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && face_tet && nF)
    e = cudaMemcpyAsync(face_tet, m->face_tet, sizeof(int2) * nF, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && face_vtx && nF)
    e = cudaMemcpyAsync(face_vtx, m->face_vtx, sizeof(int32_t) * 3 * nF, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && face_kind && nF)
    e = cudaMemcpyAsync(face_kind, m->face_kind, nF, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && face_mult && nF)
    e = cudaMemcpyAsync(face_mult, m->face_mult, sizeof(int32_t) * nF, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && face_area && nF)
    e = cudaMemcpyAsync(face_area, m->face_area, sizeof(double) * nF, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && face_centroid && nF) {
    k_face_centroid<<<grid_for(nF), kThreads, 0, s>>>(m->coord, m->face_vtx, nF, face_centroid);
    e = launched();
  }
  return cuda_status(e, "ph_mesh_faces");
}

extern "C" ph_status ph_csr_pattern(const ph_mesh* m, int32_t* rowptr, int32_t* colind, void* stream) {
  if (!m || !rowptr || (m->nnz > 0 && !colind)) return PH_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(rowptr, m->rowptr, sizeof(int32_t) * (m->L + 1), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && m->nnz)
    e = cudaMemcpyAsync(colind, m->colind, sizeof(int32_t) * m->nnz, cudaMemcpyDeviceToDevice, s);
  return cuda_status(e, "ph_csr_pattern");
}

extern "C" ph_status ph_mesh_check(ph_mesh* m, void* stream) {
  if (!m) return PH_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned bits = 0;
  cudaError_t e = cudaMemcpyAsync(&bits, m->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->status, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e, "ph_mesh_check");
  return status_from_bits(bits);
}
