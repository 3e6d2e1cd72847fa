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

#include <initializer_list>
#include <vector>


#include "element.cuh"
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

// True once an earlier kernel of this mesh recorded an error: the kernels
// after validation read ids produced by the earlier ones and must not touch
// memory through them then (the error is reported at the end of creation).
__device__ __forceinline__ bool failed(const unsigned* status) { return *status != 0; }

__device__ __forceinline__ bool valid_tri(int3 v, int64_t nC) {
  bool in = v.x >= 0 && v.y >= 0 && v.z >= 0 && v.x < nC && v.y < nC && v.z < nC;
  return in && v.x != v.y && v.x != v.z && v.y != v.z;
}

__device__ __forceinline__ int3 neumann_tri(const int32_t* nb, int64_t i) {
  return make_int3(nb[3 * i], nb[3 * i + 1], nb[3 * i + 2]);
}

// Bucket of a sorted face key (v0 < v1 < v2): the largest vertex and `sub`
// bits hashed from the other two, so a bucket holds about 2^-sub of the faces
// whose largest vertex is v2.  Hashing v0 as well as v1 matters: the faces
// around one edge (v1, v2) share both vertices, and bits of v1 alone leave
// them all in one bucket (long match scans).
__device__ __forceinline__ int64_t bucket_of(int3 s, int sub) {
  return ((int64_t)s.z << sub) | ((s.x ^ s.y) & ((1 << sub) - 1));
}

// Element geometry record of tet t (fp64; compute_geo): G_e, G_e T0^-1,
// |det E|, 1/|det E|.
__device__ __forceinline__ void tet_geom(const double* __restrict__ coord, int4 v, int64_t t,
                                         double* __restrict__ geo, unsigned* status) {
  const ph_elem::Geo G = ph_elem::compute_geo(coord, v);
  if (!ph::pos_finite(G.adet)) ph_flag(status, PH_ERR_DEGENERATE);
  double2* gg = reinterpret_cast<double2*>(geo + PH_GEO_STRIDE * t);
  gg[0] = make_double2(G.g00, G.g01);
  gg[1] = make_double2(G.g02, G.g11);
  gg[2] = make_double2(G.g12, G.g22);
  gg[3] = make_double2(G.t00, G.t01);
  gg[4] = make_double2(G.t02, G.t10);
  gg[5] = make_double2(G.t11, G.t12);
  gg[6] = make_double2(G.t20, G.t21);
  gg[7] = make_double2(G.t22, G.adet);
  gg[8] = make_double2(G.rdet, 0.0);
}

// The double-word geometry record of tet t (meshes of ph_mesh_create_dw):
// E, det E, |det E| and 1/|det E| in fp64 as in compute_geo (so |det E| and
// 1/|det E| are the fp64 record's bits), then E scaled by the power of two
// of its largest entry, G' = E'E'^T, its scale 2^kg and G'T = G' - (G' 1) 1'/4
// in double-word (dw.cuh), stored as the layout of load_geo_dw reads it.
__device__ __forceinline__ void tet_geom_dw(const double* __restrict__ coord, int4 v, int64_t t,
                                            double* __restrict__ geo, unsigned* status) {
  using namespace dw;
  const double* p0 = coord + 3 * (int64_t)v.x;
  const double* p1 = coord + 3 * (int64_t)v.y;
  const double* p2 = coord + 3 * (int64_t)v.z;
  const double* p3 = coord + 3 * (int64_t)v.w;
  double e[3][3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    e[0][d] = p1[d] - p0[d];
    e[1][d] = p2[d] - p0[d];
    e[2][d] = p3[d] - p0[d];
  }
  const double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) +
                     e[0][1] * (e[1][2] * e[2][0] - e[1][0] * e[2][2]) +
                     e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
  const double adet = ph::neg_if(det, __double2hiint(det) < 0);
  if (!ph::pos_finite(adet)) ph_flag(status, PH_ERR_DEGENERATE);
  const double rdet = ph::rcp_newton(adet);
  int kE = -1023;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int d = 0; d < 3; ++d) kE = max(kE, exponent(e[i][d]));
  f2 E[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int d = 0; d < 3; ++d) E[i][d] = from_double(e[i][d], -kE);
  f2 g[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) g[i][j] = add(add(mul(E[i][0], E[j][0]), mul(E[i][1], E[j][1])), mul(E[i][2], E[j][2]));
  const int kd = max(exponent(g[0][0].h), max(exponent(g[1][1].h), exponent(g[2][2].h)));
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) g[i][j] = ldexp(g[i][j], -kd);
  g[1][0] = g[0][1];
  g[2][0] = g[0][2];
  g[2][1] = g[1][2];
  float out[36];
  const f2 gs[6] = {g[0][0], g[0][1], g[0][2], g[1][1], g[1][2], g[2][2]};
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    out[2 * i] = gs[i].h;
    out[2 * i + 1] = gs[i].l;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const f2 q = ldexp(add(add(g[i][0], g[i][1]), g[i][2]), -2);  // row sum / 4 (exact scaling)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const f2 tij = sub(g[i][j], q);
      out[12 + 2 * (3 * i + j)] = tij.h;
      out[13 + 2 * (3 * i + j)] = tij.l;
    }
  }
  const int kg = 2 * kE + kd;
  out[30] = __int_as_float(__double2loint(adet));
  out[31] = __int_as_float(__double2hiint(adet));
  out[32] = __int_as_float(__double2loint(rdet));
  out[33] = __int_as_float(__double2hiint(rdet));
  out[34] = __int_as_float(kg);
  out[35] = __int_as_float(-2 * exponent(rdet) - (exponent(g[0][0].h) + exponent(g[1][1].h) + exponent(g[2][2].h) +
                                                  3 * kg));
  float4* o = reinterpret_cast<float4*>(geo + PH_GEO_STRIDE * t);
#pragma unroll
  for (int i = 0; i < 9; ++i) o[i] = make_float4(out[4 * i], out[4 * i + 1], out[4 * i + 2], out[4 * i + 3]);
}

// 1. histogram of face keys by bucket
__global__ void k_face_count(const int4* __restrict__ tet, int64_t nE, int64_t nC, const int32_t* __restrict__ nb,
                             int64_t nN, int sub, int32_t* __restrict__ cnt, int4* __restrict__ tet_copy,
                             unsigned* status) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < nE) {
    int4 v = tet[i];
    tet_copy[i] = v;  // the mesh's own copy of the input
    if (!valid_tet(v, nC)) { ph_flag(status, PH_ERR_ARG); return; }
#pragma unroll
    for (int k = 0; k < 4; ++k) atomicAdd(&cnt[bucket_of(sort3(local_face(v, k)), sub)], 1);
  } else if (i < nE + nN) {
    int3 f = neumann_tri(nb, i - nE);
    if (!valid_tri(f, nC)) { ph_flag(status, PH_ERR_ARG); return; }
    atomicAdd(&cnt[bucket_of(sort3(f), sub)], 1);
  }
}

// 2. scatter keys into buckets: entry = (v0, v1, v2, slot), slot = 4t+k for
//    tet faces and 4nE+i for Neumann triples.  cnt counts down to 0.  The
//    same thread then computes the tet's geometry record: the FP64-bound
//    geometry and the latency-bound atomics and scattered stores overlap in
//    the SM's warp scheduler.
__global__ void k_face_fill(const int4* __restrict__ tet, int64_t nE, int64_t nC, const int32_t* __restrict__ nb,
                            int64_t nN, int sub, const int32_t* __restrict__ start, int32_t* __restrict__ cnt,
                            int4* __restrict__ entries, int32_t* __restrict__ mate, const double* __restrict__ coord,
                            double* __restrict__ geo, bool geo_dw, unsigned* status) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (failed(status)) return;
  if (i < nE) {
    int4 v = tet[i];
    if (!valid_tet(v, nC)) return;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      int3 s = sort3(local_face(v, k));
      const int64_t b = bucket_of(s, sub);
      int pos = start[b] + atomicSub(&cnt[b], 1) - 1;
      entries[pos] = make_int4(s.x, s.y, s.z, (int)(4 * i + k));
    }
    reinterpret_cast<int4*>(mate)[i] = make_int4(-1, -1, -1, -1);  // no mate yet (boundary)
    if (geo_dw) tet_geom_dw(coord, v, i, geo, status);
    else tet_geom(coord, v, i, geo, status);
  } else if (i < nE + nN) {
    int3 f = neumann_tri(nb, i - nE);
    if (!valid_tri(f, nC)) return;
    int3 s = sort3(f);
    const int64_t b = bucket_of(s, sub);
    int pos = start[b] + atomicSub(&cnt[b], 1) - 1;
    entries[pos] = make_int4(s.x, s.y, s.z, (int)i + 3 * (int)nE);  // slot 4nE + (i - nE)
  }
}

// Outcome of one entry's scan: a tet entry records its mate (and its mate's
// mate) or -2 for a Neumann triple; errors as in k_face_match.
__device__ __forceinline__ void settle_entry(int4 e, int ntet, int nt, int nn, int tm, int32_t* __restrict__ mate,
                                             unsigned* status) {
  if (e.w < ntet) {
    if (nt + nn >= 2) ph_flag(status, nn > 0 ? PH_ERR_ARG : PH_ERR_NONMANIFOLD);
    if (nt == 1) {
      mate[e.w] = tm;
      mate[tm] = e.w;
    } else if (nn == 1) {
      mate[e.w] = -2;
    }
  } else {
    if (nt != 1 || nn != 0) ph_flag(status, PH_ERR_ARG);
    else mate[tm] = -2;
  }
}

// k is an entry of e's bucket (same largest vertex) or the sentinel (-1, ...),
// which equals no entry
__device__ __forceinline__ void count_match(int4 k, int4 e, int ntet, int& nt, int& nn, int& tm) {
  if (k.x == e.x && k.y == e.y) {
    if (k.w < ntet) { ++nt; tm = k.w; } else { ++nn; }
  }
}

// 3. match equal keys inside a bucket.  A tet entry compares itself with the
//    LATER entries of its bucket only and writes both mates of a pair, so each
//    pair is found once (a second match marks a face in three tets, or a
//    Neumann triple on an interior face); Neumann entries (boundary only, few)
//    scan the whole bucket, themselves included (one Neumann hit taken off),
//    and must match exactly one tet entry.  Each thread takes two entries, i
//    and i + half, and scans their buckets in lockstep: two independent chains
//    of loads in flight per thread.  The kernel issues instructions at close
//    to the SM's rate, so the loop carries no more than the loads and
//    compares; the bucket hash keeps the scans short.
__global__ void k_face_match(const int4* __restrict__ entries, int64_t nent, const int32_t* __restrict__ start,
                             int sub, int64_t nE, int32_t* __restrict__ mate, unsigned* status) {
  const int64_t half = (nent + 1) >> 1;
  const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i0 >= half || failed(status)) return;
  const int64_t i1 = i0 + half;
  const bool has1 = i1 < nent;
  const int ntet = (int)(4 * nE);  // slots are int32
  const int4 none = make_int4(-1, -1, -1, -1);
  const int4 e0 = entries[i0];
  const int4 e1 = has1 ? entries[i1] : none;
  const int64_t b0 = bucket_of(make_int3(e0.x, e0.y, e0.z), sub);
  const int64_t b1 = has1 ? bucket_of(make_int3(e1.x, e1.y, e1.z), sub) : 0;
  const int end0 = start[b0 + 1], end1 = has1 ? start[b1 + 1] : 0;
  // tet entries scan the later entries of their bucket, Neumann entries all of it
  const bool nm0 = e0.w >= ntet, nm1 = has1 && e1.w >= ntet;
  int j0 = nm0 ? start[b0] : (int)i0 + 1;
  int j1 = has1 ? (nm1 ? start[b1] : (int)i1 + 1) : 0;
  int nt0 = 0, nn0 = nm0 ? -1 : 0, tm0 = -1, nt1 = 0, nn1 = nm1 ? -1 : 0, tm1 = -1;
  while (j0 < end0 || j1 < end1) {
    const int4 k0 = j0 < end0 ? entries[j0] : none;
    const int4 k1 = j1 < end1 ? entries[j1] : none;
    count_match(k0, e0, ntet, nt0, nn0, tm0);
    count_match(k1, e1, ntet, nt1, nn1, tm1);
    ++j0;
    ++j1;
  }
  settle_entry(e0, ntet, nt0, nn0, tm0, mate, status);
  if (has1) settle_entry(e1, ntet, nt1, nn1, tm1, mate, status);
}

// 4. face bases: an exclusive scan of the number of first occurrences per tet,
//    which the scan itself counts from the mates (exclusive_scan's `mates`).
using ph::first_occurrence;

__device__ __forceinline__ int first_rank(int4 m, int s0, int k) {
  int r = 0;
  if (k > 0) r += first_occurrence(m.x, s0);
  if (k > 1) r += first_occurrence(m.y, s0 + 1);
  if (k > 2) r += first_occurrence(m.z, s0 + 2);
  return r;
}

// Outputs of tet t, given its tuple v, mates m, face base fb and, for each
// face it does not own, its owner's mates om[k] and face base ofb[k].
__device__ __forceinline__ void emit_tet(int64_t t, int4 v, int4 m, int fb, const int4 om[4], const int ofb[4],
                                         int64_t nF, int4* __restrict__ tface, int2* __restrict__ face_tet,
                                         int32_t* __restrict__ face_vtx, int8_t* __restrict__ face_kind,
                                         int32_t* __restrict__ flag, int32_t* __restrict__ mult_iota,
                                         int4* __restrict__ tmult, int32_t* __restrict__ rowlen) {
  const int s0 = (int)(4 * t);
  int out[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int mk = comp(m, k);
    if (first_occurrence(mk, s0 + k)) {
      const int F = fb + first_rank(m, s0, k);
      out[k] = F;
      face_tet[F] = make_int2((int)t, mk >= 0 ? (mk >> 2) : -1);
      const int3 lf = local_face(v, k);
      face_vtx[3 * (int64_t)F] = lf.x;
      face_vtx[3 * (int64_t)F + 1] = lf.y;
      face_vtx[3 * (int64_t)F + 2] = lf.z;
      const int kind = mk >= 0 ? 0 : (mk == -1 ? 1 : 2);
      face_kind[F] = (int8_t)kind;
      if (flag) flag[F] = kind != 2;      // Neumann faces present: multipliers by a scan of the flags
      if (mult_iota) {                    // none: l(F) = F
        mult_iota[F] = F;
        rowlen[F] = mk >= 0 ? 7 : 4;
        if (F + 1 == nF) rowlen[F + 1] = 0;  // the scan reads one entry past the last row
      }
    } else {
      const int t2 = mk >> 2, k2 = mk & 3;
      out[k] = (int)((unsigned)(ofb[k] + first_rank(om[k], 4 * t2, k2)) | 0x80000000u);
    }
  }
  tface[t] = make_int4(out[0], out[1], out[2], out[3]);
  if (mult_iota) {
    int o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) o[k] = (int)((unsigned)(out[k] & PH_ID_MASK) | (comp(m, k) < 0 ? PH_BND_BIT : 0u));
    tmult[t] = make_int4(o[0], o[1], o[2], o[3]);
  }
}

// The owner's mates and face base for each face of a tet it does not own.
__device__ __forceinline__ void load_owners(int64_t t, int4 m, const int4* __restrict__ mate4,
                                            const int32_t* __restrict__ fbase, int4 om[4], int ofb[4]) {
  const int s0 = (int)(4 * t);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int mk = comp(m, k);
    if (!first_occurrence(mk, s0 + k)) {
      om[k] = mate4[mk >> 2];
      ofb[k] = fbase[mk >> 2];
    }
  }
}

// 5. per tet: face ids, T+/T-, T+'s tuple, kind and non-Neumann flag of the
//    faces it owns (first occurrences).  Without Neumann faces (mult_iota
//    given) every face has a multiplier, l(F) = F, so the tet also writes its
//    slots' multiplier ids and, for the faces it owns, the row length 1 + 3
//    per tet of the face (7 interior, 4 boundary); k_tet_mult is not needed.
//    Each thread takes two tets, t and t + half, and issues all their loads
//    before using any (its warps mostly wait on loads).
__global__ void k_face_emit(const int4* __restrict__ tet, int64_t nE, const int4* __restrict__ mate4,
                            const int32_t* __restrict__ fbase, int4* __restrict__ tface, int2* __restrict__ face_tet,
                            int32_t* __restrict__ face_vtx, int8_t* __restrict__ face_kind,
                            int32_t* __restrict__ flag, int32_t* __restrict__ mult_iota, int4* __restrict__ tmult,
                            int32_t* __restrict__ rowlen, const unsigned* status) {
  const int64_t half = (nE + 1) >> 1;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t0 >= half || failed(status)) return;
  const int64_t t1 = t0 + half;
  const bool has1 = t1 < nE;
  const int nF = fbase[nE];
  const int4 v0 = tet[t0], m0 = mate4[t0];
  const int fb0 = fbase[t0];
  const int4 v1 = has1 ? tet[t1] : make_int4(0, 0, 0, 0);
  const int4 m1 = has1 ? mate4[t1] : make_int4(-1, -1, -1, -1);
  const int fb1 = has1 ? fbase[t1] : 0;
  int4 om0[4], om1[4];
  int ofb0[4], ofb1[4];
  load_owners(t0, m0, mate4, fbase, om0, ofb0);
  if (has1) load_owners(t1, m1, mate4, fbase, om1, ofb1);
  emit_tet(t0, v0, m0, fb0, om0, ofb0, nF, tface, face_tet, face_vtx, face_kind, flag, mult_iota, tmult, rowlen);
  if (has1)
    emit_tet(t1, v1, m1, fb1, om1, ofb1, nF, tface, face_tet, face_vtx, face_kind, flag, mult_iota, tmult, rowlen);
}

// face area 1/2 |(P_z - P_x) x (P_y - P_x)|
__device__ __forceinline__ void face_area(const double* __restrict__ coord, const int32_t* __restrict__ face_vtx,
                                          int64_t F, double* __restrict__ area) {
  const double* x = coord + 3 * (int64_t)face_vtx[3 * F];
  const double* y = coord + 3 * (int64_t)face_vtx[3 * F + 1];
  const double* z = coord + 3 * (int64_t)face_vtx[3 * F + 2];
  double u0 = z[0] - x[0], u1 = z[1] - x[1], u2 = z[2] - x[2];
  double v0 = y[0] - x[0], v1 = y[1] - x[1], v2 = y[2] - x[2];
  double cx = u1 * v2 - u2 * v1, cy = u2 * v0 - u0 * v2, cz = u0 * v1 - u1 * v0;
  area[F] = ph::half_sqrt(cx * cx + cy * cy + cz * cz);
}

// Neumann faces get no multiplier.  Face counts are read on the device
// (d_tot[0] = nF), the grid covers the upper bound.
__global__ void k_mult_fix(int32_t* __restrict__ face_mult, const int8_t* __restrict__ face_kind,
                           const int64_t* __restrict__ d_tot, int64_t nFmax, const unsigned* status) {
  int64_t F = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (F >= nFmax || F >= d_tot[0] || failed(status)) return;
  if (face_kind[F] == 2) face_mult[F] = -1;
}

// 7. per-slot multiplier ids and row lengths: row l(F) = 1 + sum over F's
//    tets of (non-Neumann faces of the tet) - 1.
__global__ void k_tet_mult(const int4* __restrict__ tface, int64_t nE, const int32_t* __restrict__ face_mult,
                           const int2* __restrict__ face_tet, int4* __restrict__ tmult, int32_t* __restrict__ rowlen,
                           const unsigned* status) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nE || failed(status)) return;
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

// The other three local faces of a tet, m != k ascending, as multiplier ids
// (PH_NO_MULT, which sorts last, for Neumann faces or no tet).
__device__ __forceinline__ void other_mults(int4 tm, int k, int& o0, int& o1, int& o2) {
  int id[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int mj = comp(tm, j);
    id[j] = mj == PH_NO_MULT ? PH_NO_MULT : (mj & PH_ID_MASK);
  }
  o0 = k == 0 ? id[1] : id[0];
  o1 = k <= 1 ? id[2] : id[1];
  o2 = k <= 2 ? id[3] : id[2];
}

__device__ __forceinline__ void cswap(int& a, int& b) {
  const int lo = min(a, b), hi = max(a, b);
  a = lo;
  b = hi;
}

// number of entries of c[0..7) below x (the rank of x among distinct ids)
__device__ __forceinline__ int rank7(const int c[7], int x) {
  int r = 0;
#pragma unroll
  for (int i = 0; i < 7; ++i) r += c[i] < x;
  return r;
}

// 8. column indices of each row (ascending), the diagonal position, and each
//    slot's scatter positions: tpos = diagonal, trel = rank offsets of the
//    other three local faces (4-bit two's complement, m != k ascending).
//    Row l(F) holds l(F) and the other non-Neumann faces of F's one or two
//    tets (all distinct): 7 candidates with PH_NO_MULT for absent ones, put in
//    order by a 16-comparator sorting network, all in registers.  The thread
//    first computes the face's area (FP64), which overlaps the gathers.
__global__ void k_row_fill(const int2* __restrict__ face_tet, const int4* __restrict__ tface,
                           const int4* __restrict__ tmult, const int32_t* __restrict__ face_mult,
                           const int64_t* __restrict__ d_tot, int64_t nFmax,
                           const int32_t* __restrict__ rowptr, int32_t* __restrict__ colind,
                           int32_t* __restrict__ rowdiag, int32_t* __restrict__ tpos,
                           unsigned short* __restrict__ trel, const double* __restrict__ coord,
                           const int32_t* __restrict__ face_vtx, double* __restrict__ area, unsigned* status) {
  const int64_t F = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (F >= nFmax || F >= d_tot[0] || failed(status)) return;
  face_area(coord, face_vtx, F, area);
  const int l = face_mult[F];
  if (l < 0) return;
  const int2 ft = face_tet[F];
  const int T[2] = {ft.x, ft.y};
  int k[2] = {0, 0};
  int o[2][3];
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    o[side][0] = o[side][1] = o[side][2] = PH_NO_MULT;
    if (T[side] < 0) continue;
    const int4 tf = tface[T[side]], tm = tmult[T[side]];
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if ((comp(tf, j) & PH_ID_MASK) == F) k[side] = j;
    other_mults(tm, k[side], o[side][0], o[side][1], o[side][2]);
  }
  int c[7] = {l, o[0][0], o[0][1], o[0][2], o[1][0], o[1][1], o[1][2]};
  cswap(c[0], c[6]); cswap(c[2], c[3]); cswap(c[4], c[5]);
  cswap(c[0], c[2]); cswap(c[1], c[4]); cswap(c[3], c[6]);
  cswap(c[0], c[1]); cswap(c[2], c[5]); cswap(c[3], c[4]);
  cswap(c[1], c[2]); cswap(c[4], c[6]);
  cswap(c[2], c[3]); cswap(c[4], c[5]);
  cswap(c[1], c[2]); cswap(c[3], c[4]); cswap(c[5], c[6]);
  const int n = 7 - ((c[0] == PH_NO_MULT) + (c[1] == PH_NO_MULT) + (c[2] == PH_NO_MULT) + (c[3] == PH_NO_MULT) +
                     (c[4] == PH_NO_MULT) + (c[5] == PH_NO_MULT) + (c[6] == PH_NO_MULT));
  const int base = rowptr[l];
  if (rowptr[l + 1] - base != n) { ph_flag(status, PH_ERR_ARG); return; }
#pragma unroll
  for (int i = 0; i < 7; ++i)
    if (i < n) colind[base + i] = c[i];
  const int rl = rank7(c, l);
  rowdiag[l] = base + rl;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    if (T[side] < 0) continue;
    unsigned bits = 0;
#pragma unroll
    for (int idx = 0; idx < 3; ++idx) {
      const int lm = o[side][idx];
      if (lm != PH_NO_MULT) bits |= ((unsigned)(rank7(c, lm) - rl) & 0xFu) << (4 * idx);
    }
    tpos[4 * (int64_t)T[side] + k[side]] = base + rl;
    trel[4 * (int64_t)T[side] + k[side]] = (unsigned short)bits;
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
  if (m->shared) {
    if (m->shared->refs.fetch_sub(1) == 1) {
      free_async(m->shared->arena, s);
      free_async(m->shared->extra, s);
      delete m->shared;
    }
  } else {
    free_async(m->arena, s);
  }
  delete m;
}

// Offsets of the problems of a batched build (the union mesh of
// ph_mesh_create_batch), one thread per problem.  Problem p owns tets
// [toff[p], toff[p+1]); its faces, multipliers and CSR entries are
// contiguous, and start at: the face of its first tet's first local face
// (always a first occurrence), the multiplier of the first non-Neumann face at
// or after it (Neumann faces have none; the walk may run into the next
// problem's faces, whose first multiplier is then this problem's end, which is
// also its start when it has no multiplier), and that row's first CSR entry.
// An empty problem gets -1 (the host takes the next problem's offsets).
__global__ void k_batch_offsets(const int4* __restrict__ tface, const int32_t* __restrict__ face_mult,
                                const int32_t* __restrict__ rowptr, const int64_t* __restrict__ d_tot,
                                const int64_t* __restrict__ toff, int32_t n, long long* __restrict__ out,
                                const unsigned* status) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  long long f0 = -1, m0 = -1, z0 = -1;
  if (toff[p + 1] > toff[p] && !failed(status)) {
    const int64_t nF = d_tot[0], L = d_tot[1];
    f0 = tface[toff[p]].x & PH_ID_MASK;
    int64_t F = f0;
    while (F < nF && face_mult[F] < 0) ++F;
    m0 = F < nF ? face_mult[F] : L;
    z0 = rowptr[m0];
  }
  out[3 * p] = f0;
  out[3 * p + 1] = m0;
  out[3 * p + 2] = z0;
}

// Hook of a batched build: the per-problem offsets, computed before the
// build's one synchronisation and read with it.
struct BatchCounts {
  const int64_t* d_toff;  // n + 1 tet offsets (device)
  int32_t n;
  long long* d_counts;  // 3n: first face, multiplier, CSR entry of each problem
  long long* h_counts;  // 3n (host)
};

// Synchronise and read n device int64 counters and the status word.
static ph_status read_counters(const int64_t* d_tot, int n, unsigned* d_status, cudaStream_t s, int64_t* tot,
                               unsigned* status) {
  cudaError_t e = cudaMemcpyAsync(tot, d_tot, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(status, d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return cuda_status(e, "mesh_create sync");
}

#define PH_TRY(expr)                    \
  do {                                  \
    st = (expr);                        \
    if (st != PH_OK) goto fail;         \
  } while (0)
#define PH_CU(expr, what) PH_TRY(cuda_status((expr), what))

static ph_status mesh_build(const double* coord, int64_t nC, const int32_t* tet, int64_t nE, const int32_t* neumann,
                            int64_t nN, cudaStream_t s, ph_mesh** out, const BatchCounts* bc, bool dw = false);

extern "C" ph_status ph_mesh_create(const double* coord, int64_t nC, const int32_t* tet, int64_t nE,
                                    const int32_t* neumann, int64_t nN, void* stream, ph_mesh** out) {
  return mesh_build(coord, nC, tet, nE, neumann, nN, (cudaStream_t)stream, out, nullptr);
}

extern "C" ph_status ph_mesh_create_dw(const double* coord, int64_t nC, const int32_t* tet, int64_t nE,
                                       const int32_t* neumann, int64_t nN, void* stream, ph_mesh** out) {
  return mesh_build(coord, nC, tet, nE, neumann, nN, (cudaStream_t)stream, out, nullptr, true);
}

static ph_status mesh_build(const double* coord, int64_t nC, const int32_t* tet, int64_t nE, const int32_t* neumann,
                            int64_t nN, cudaStream_t s, ph_mesh** out, const BatchCounts* bc, bool dw) {
  if (!out) return PH_ERR_ARG;
  *out = nullptr;
  if (nE < 0 || nC < 0 || nN < 0 || (nE > 0 && (!coord || !tet)) || (nN > 0 && !neumann)) return PH_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(tet) & 15u) != 0) return PH_ERR_ARG;  // read as int4
  // Face arrays are sized by nFmax = 4 nE + nN >= nF and the CSR columns by
  // nFmax + 12 nE >= nnz, so the whole construction is enqueued at once and
  // synchronises once, at the end; int32 ids and CSR positions bound the size.
  const int64_t nFmax = 4 * nE + nN, nnzmax = nFmax + 12 * nE;
  if (nnzmax >= ((int64_t)1 << 31) - 1 || nC >= ((int64_t)1 << 31) - 1) return PH_ERR_OVERFLOW;
  ph_status st = PH_OK;  // everything runs in order on the caller's stream s
  // face-key buckets: 4 per largest vertex while the bucket ids stay below 2^31
  // (finer buckets shorten the match scans but cost more in the scattered
  // fill and the bucket scan than they save)
  const int sub = nC < ((int64_t)1 << 28) ? 2 : 0;
  const int64_t nb = (nC << sub) + 1;
  const int64_t nent = nFmax;
  const unsigned gF = grid_for(nFmax + 1);
  ph_mesh* m = new ph_mesh();
  memset(m, 0, sizeof *m);
  int64_t tot[3] = {0, 0, 0};
  unsigned bits = 0;
  // Two allocations: the mesh's arrays, and the scratch of the build (its
  // first part zeroed by one memset).  Few host calls keep the GPU fed.
  Carve mc, sc;
  const size_t o_status = mc.take<unsigned>(1), o_coord = mc.take<double>(3 * nC), o_tet = mc.take<int4>(nE);
  const size_t o_geo = mc.take<double>(PH_GEO_STRIDE * nE), o_tface = mc.take<int4>(nE);
  const size_t o_tmult = mc.take<int4>(nE), o_tpos = mc.take<int4>(nE), o_trel = mc.take<ushort4>(nE);
  const size_t o_ftet = mc.take<int2>(nFmax), o_fvtx = mc.take<int32_t>(3 * nFmax);
  const size_t o_fkind = mc.take<int8_t>(nFmax), o_fmult = mc.take<int32_t>(nFmax + 1);
  const size_t o_farea = mc.take<double>(nFmax), o_rowptr = mc.take<int32_t>(nFmax + 1);
  const size_t o_colind = mc.take<int32_t>(nnzmax), o_rowdiag = mc.take<int32_t>(nFmax);
  // scratch: zeroed part first
  const size_t o_tot = sc.take<int64_t>(3), o_cnt = sc.take<int32_t>(nb);
  const size_t o_s1 = sc.take<unsigned long long>(scan_state_words(nb));
  const size_t o_s2 = sc.take<unsigned long long>(scan_state_words(nE + 1));
  const size_t o_s3 = sc.take<unsigned long long>(scan_state_words(nFmax + 1));
  const size_t o_s4 = sc.take<unsigned long long>(scan_state_words(nFmax + 1));
  const size_t o_rowlen = sc.take<int32_t>(nN > 0 || nE == 0 ? nFmax + 1 : 0);  // else written by k_face_emit
  const size_t o_flag = sc.take<int32_t>(nN > 0 ? nFmax + 1 : 0);
  const size_t zero_bytes = sc.bytes;
  const size_t o_start = sc.take<int32_t>(nb), o_entries = sc.take<int4>(nent), o_mate = sc.take<int32_t>(4 * nE);
  const size_t o_newc = sc.take<int32_t>(nE + 1);
  const size_t o_rowlen2 = sc.take<int32_t>(nN > 0 || nE == 0 ? 0 : nFmax + 1);
  void* scratch = nullptr;
  PH_CU(cudaGetDevice(&m->device), "cudaGetDevice");
  m->nE = nE;
  m->nC = nC;
  PH_CU(alloc_bytes(&m->arena, mc.bytes, s), "alloc mesh");
  PH_CU(alloc_bytes(&scratch, sc.bytes, s), "alloc scratch");
  {
    void* A = m->arena;
    m->status = Carve::at<unsigned>(A, o_status);
    m->coord = Carve::at<double>(A, o_coord);
    m->tet = Carve::at<int4>(A, o_tet);
    m->geo = Carve::at<double>(A, o_geo);
    m->tface = Carve::at<int4>(A, o_tface);
    m->tmult = Carve::at<int4>(A, o_tmult);
    m->tpos = Carve::at<int4>(A, o_tpos);
    m->trel = Carve::at<ushort4>(A, o_trel);
    m->face_tet = Carve::at<int2>(A, o_ftet);
    m->face_vtx = Carve::at<int32_t>(A, o_fvtx);
    m->face_kind = Carve::at<int8_t>(A, o_fkind);
    m->face_mult = Carve::at<int32_t>(A, o_fmult);
    m->face_area = Carve::at<double>(A, o_farea);
    m->rowptr = Carve::at<int32_t>(A, o_rowptr);
    m->colind = Carve::at<int32_t>(A, o_colind);
    m->rowdiag = Carve::at<int32_t>(A, o_rowdiag);
  }
  {
  int64_t* d_tot = Carve::at<int64_t>(scratch, o_tot);  // [0] nF, [1] L, [2] nnz
  int32_t* cnt = Carve::at<int32_t>(scratch, o_cnt);
  int32_t* newc = Carve::at<int32_t>(scratch, o_newc);
  int32_t* start = Carve::at<int32_t>(scratch, o_start);
  int4* entries = Carve::at<int4>(scratch, o_entries);
  int32_t* mate = Carve::at<int32_t>(scratch, o_mate);
  int32_t* flag = nN > 0 ? Carve::at<int32_t>(scratch, o_flag) : nullptr;
  int32_t* rowlen = Carve::at<int32_t>(scratch, (nN > 0 || nE == 0) ? o_rowlen : o_rowlen2);
  unsigned long long* st1 = Carve::at<unsigned long long>(scratch, o_s1);
  unsigned long long* st2 = Carve::at<unsigned long long>(scratch, o_s2);
  unsigned long long* st3 = Carve::at<unsigned long long>(scratch, o_s3);
  unsigned long long* st4 = Carve::at<unsigned long long>(scratch, o_s4);
  PH_CU(cudaMemsetAsync(scratch, 0, zero_bytes, s), "memset");
  PH_CU(cudaMemsetAsync(m->status, 0, sizeof(unsigned), s), "memset");
  if (nC > 0) PH_CU(cudaMemcpyAsync(m->coord, coord, sizeof(double) * 3 * nC, cudaMemcpyDeviceToDevice, s), "copy");

  // --- faces: bucket the keys, match them, number the faces ----------------
  if (nent > 0) {
    KernelTimer kt("k_face_count", s, 2);
    k_face_count<<<grid_for(nE + nN), kThreads, 0, s>>>(reinterpret_cast<const int4*>(tet), nE, nC, neumann, nN,
                                                        sub, cnt, m->tet, m->status);
    PH_CU(launched(), "k_face_count");
  }
  PH_TRY(exclusive_scan(cnt, start, nb, d_tot, s, m->status, nullptr, 0, st1));
  if (nent > 0) {
    {
      KernelTimer kt("k_face_fill", s, 2);
      k_face_fill<<<grid_for(nE + nN), kThreads, 0, s>>>(m->tet, nE, nC, neumann, nN, sub, start, cnt, entries,
                                                         mate, m->coord, m->geo, dw, m->status);
      PH_CU(launched(), "k_face_fill");
    }
    {
      KernelTimer kt("k_face_match", s, 2);
      k_face_match<<<grid_for((nent + 1) / 2), kThreads, 0, s>>>(entries, nent, start, sub, nE, mate, m->status);
      PH_CU(launched(), "k_face_match");
    }
  }
  // face bases: the scan counts each tet's first occurrences from the mates
  PH_TRY(exclusive_scan(nullptr, newc, nE + 1, d_tot, s, m->status, nullptr, 0, st2,
                        reinterpret_cast<const int4*>(mate), nE));  // nF -> d_tot[0]
  if (nE > 0) {
    KernelTimer kt("k_face_emit", s, 2);
    k_face_emit<<<grid_for((nE + 1) / 2), kThreads, 0, s>>>(
        m->tet, nE, reinterpret_cast<int4*>(mate), newc, m->tface, m->face_tet, m->face_vtx, m->face_kind, flag,
        nN > 0 ? nullptr : m->face_mult, m->tmult, rowlen, m->status);
    PH_CU(launched(), "k_face_emit");
  }

  // --- multipliers and CSR pattern (rows sized by nFmax >= L) ---------------
  if (nN > 0) {
    PH_TRY(exclusive_scan(flag, m->face_mult, nFmax + 1, d_tot + 1, s, m->status, d_tot, 1, st3));  // L -> d_tot[1]
    k_mult_fix<<<gF, kThreads, 0, s>>>(m->face_mult, m->face_kind, d_tot, nFmax, m->status);
    PH_CU(launched(), "k_mult_fix");
    if (nE > 0) {
      k_tet_mult<<<grid_for(nE), kThreads, 0, s>>>(m->tface, nE, m->face_mult, m->face_tet, m->tmult, rowlen,
                                                   m->status);
      PH_CU(launched(), "k_tet_mult");
    }
  } else {  // every face has a multiplier (k_face_emit wrote them, the slots' ids and the row lengths): L = nF
    PH_CU(cudaMemcpyAsync(d_tot + 1, d_tot, sizeof(int64_t), cudaMemcpyDeviceToDevice, s), "copy");
  }
  PH_TRY(exclusive_scan(rowlen, m->rowptr, nFmax + 1, d_tot + 2, s, m->status, d_tot + 1, 1, st4));  // nnz

  // --- CSR columns and scatter positions (slots without a multiplier are never read)
  if (nFmax > 0) {
    KernelTimer kt("k_row_fill", s, 2);
    k_row_fill<<<gF, kThreads, 0, s>>>(m->face_tet, m->tface, m->tmult, m->face_mult, d_tot, nFmax, m->rowptr,
                                       m->colind, m->rowdiag, reinterpret_cast<int32_t*>(m->tpos),
                                       reinterpret_cast<unsigned short*>(m->trel), m->coord, m->face_vtx,
                                       m->face_area, m->status);
    PH_CU(launched(), "k_row_fill");
  }
  if (bc && bc->n > 0) {  // per-problem offsets of a batched build
    k_batch_offsets<<<grid_for(bc->n), kThreads, 0, s>>>(m->tface, m->face_mult, m->rowptr, d_tot, bc->d_toff, bc->n,
                                                         bc->d_counts, m->status);
    PH_CU(launched(), "k_batch_offsets");
    PH_CU(cudaMemcpyAsync(bc->h_counts, bc->d_counts, sizeof(long long) * 3 * bc->n, cudaMemcpyDeviceToHost, s),
          "copy");
  }
  // the one synchronisation: counts and the first error of any kernel
  PH_TRY(read_counters(d_tot, 3, m->status, s, tot, &bits));
  }
  free_async(scratch, s);
  scratch = nullptr;
  if (bits) { st = status_from_bits(bits); goto fail; }
  m->nF = tot[0];
  m->L = tot[1];
  m->nnz = tot[2];
  // face kinds: every interior face has two slots and a boundary face one,
  // so 4 nE = 2 nFi + (nF - nFi); Neumann faces are the ones without multiplier
  m->nFi = 4 * nE - m->nF;
  m->nFn = m->nF - m->L;
  m->nFd = m->nF - m->nFi - m->nFn;
  m->geo_dw = dw;
  *out = m;
  return PH_OK;

fail:
  free_async(scratch, s);
  mesh_free(m, s);
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

// ---------------------------------------------------------------------------
// Batched build: n meshes at once.  Their disjoint union (vertex ids of
// problem p shifted by the vertices of the problems before it) is built as one
// mesh: faces of different problems never match, and the first-occurrence
// numbering of the union, restricted to problem p, is p's own numbering
// shifted by the faces of the problems before it (p's tets are consecutive);
// the same holds for multipliers, CSR rows and CSR entries.  So one build
// gives every problem's connectivity; a rebase pass then subtracts each
// problem's offsets, and the per-problem meshes are views into the union's
// memory with local ids, bit-identical to building each alone.
// ---------------------------------------------------------------------------
namespace {

// Offsets of problem p in the union (device, n + 1 entries each).
struct UnionOffsets {
  const int64_t *toff, *voff, *foff, *moff, *zoff;
  int32_t n;
};

// last p with off[p] <= i (off ascending, off[0] = 0)
__device__ __forceinline__ int problem_of(const int64_t* __restrict__ off, int32_t n, int64_t i) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct UnionSources {
  const int32_t* tet;  // problem's tets (nE_p x 4)
  const int32_t* nb;   // problem's Neumann triples or null
};

// union tets and Neumann triples: problem p's ids shifted by voff[p].  An id
// outside [0, nC_p) would land on another problem's vertex, so it becomes -1,
// which the union build rejects (PH_ERR_ARG).
__device__ __forceinline__ int shift_vertex(int x, int v, int nv) { return (x >= 0 && x < nv) ? x + v : -1; }

__global__ void k_union_inputs(const UnionSources* __restrict__ src, const int64_t* __restrict__ toff,
                               const int64_t* __restrict__ noff, const int64_t* __restrict__ voff, int32_t n,
                               int64_t nE, int64_t nN, int4* __restrict__ tet_u, int32_t* __restrict__ nb_u) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < nE) {
    const int p = problem_of(toff, n, i);
    const int v = (int)voff[p], nv = (int)(voff[p + 1] - voff[p]);
    const int4 t = reinterpret_cast<const int4*>(src[p].tet)[i - toff[p]];
    tet_u[i] = make_int4(shift_vertex(t.x, v, nv), shift_vertex(t.y, v, nv), shift_vertex(t.z, v, nv),
                         shift_vertex(t.w, v, nv));
  } else if (i < nE + nN) {
    const int64_t j = i - nE;
    const int p = problem_of(noff, n, j);
    const int v = (int)voff[p], nv = (int)(voff[p + 1] - voff[p]);
    const int64_t k = j - noff[p];
    nb_u[3 * j] = shift_vertex(src[p].nb[3 * k], v, nv);
    nb_u[3 * j + 1] = shift_vertex(src[p].nb[3 * k + 1], v, nv);
    nb_u[3 * j + 2] = shift_vertex(src[p].nb[3 * k + 2], v, nv);
  }
}

__device__ __forceinline__ int shift_id(int x, int64_t off) {  // keep bit 31 (sigma / Dirichlet mark)
  return (int)(((unsigned)x & 0x80000000u) | (unsigned)((x & PH_ID_MASK) - (int)off));
}

// per tet: local vertex ids, face ids, multiplier ids, CSR positions
__global__ void k_rebase_tets(UnionOffsets o, int64_t nE, int4* __restrict__ tet, int4* __restrict__ tface,
                              int4* __restrict__ tmult, int4* __restrict__ tpos) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nE) return;
  const int p = problem_of(o.toff, o.n, t);
  const int v = (int)o.voff[p], z = (int)o.zoff[p];
  const int64_t f = o.foff[p], mo = o.moff[p];
  const int4 a = tet[t];
  tet[t] = make_int4(a.x - v, a.y - v, a.z - v, a.w - v);
  const int4 b = tface[t];
  tface[t] = make_int4(shift_id(b.x, f), shift_id(b.y, f), shift_id(b.z, f), shift_id(b.w, f));
  const int4 c = tmult[t];
  int cm[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (cm[k] != PH_NO_MULT) cm[k] = shift_id(cm[k], mo);
  tmult[t] = make_int4(cm[0], cm[1], cm[2], cm[3]);
  const int4 d = tpos[t];  // positions of Neumann slots are never read
  tpos[t] = make_int4(d.x - z, d.y - z, d.z - z, d.w - z);
}

// per face: local T+/T-, vertex ids and multiplier id
__global__ void k_rebase_faces(UnionOffsets o, int64_t nF, int2* __restrict__ face_tet,
                               int32_t* __restrict__ face_vtx, int32_t* __restrict__ face_mult) {
  const int64_t F = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (F >= nF) return;
  const int p = problem_of(o.foff, o.n, F);
  const int t0 = (int)o.toff[p], v = (int)o.voff[p];
  const int2 ft = face_tet[F];
  face_tet[F] = make_int2(ft.x - t0, ft.y < 0 ? -1 : ft.y - t0);
  face_vtx[3 * F] -= v;
  face_vtx[3 * F + 1] -= v;
  face_vtx[3 * F + 2] -= v;
  const int l = face_mult[F];
  if (l >= 0) face_mult[F] = l - (int)o.moff[p];
}

// per multiplier row: the problem's own row pointers (problem p's L_p + 1
// entries at rowptr_b + moff[p] + p) and diagonal positions
__global__ void k_rebase_rows(UnionOffsets o, int64_t L, const int32_t* __restrict__ rowptr,
                              int32_t* __restrict__ rowptr_b, int32_t* __restrict__ rowdiag) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= L + o.n) return;
  if (l < L) {
    const int p = problem_of(o.moff, o.n, l);
    const int z = (int)o.zoff[p];
    rowptr_b[l + p] = rowptr[l] - z;
    rowdiag[l] -= z;
  } else {  // the closing entry of problem p: its nnz
    const int p = (int)(l - L);
    rowptr_b[o.moff[p + 1] + p] = (int)(o.zoff[p + 1] - o.zoff[p]);
  }
}

// per CSR entry: local column ids
__global__ void k_rebase_cols(UnionOffsets o, int64_t nnz, int32_t* __restrict__ colind) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= nnz) return;
  colind[j] -= (int)o.moff[problem_of(o.zoff, o.n, j)];
}

}  // namespace

extern "C" ph_status ph_mesh_create_batch(int32_t n, const double* const* coord, const int64_t* nC,
                                          const int32_t* const* tet, const int64_t* nE,
                                          const int32_t* const* neumann, const int64_t* nN, void* stream,
                                          ph_mesh** out) {
  if (n < 0 || !out || (n > 0 && (!coord || !nC || !tet || !nE))) return PH_ERR_ARG;
  for (int32_t p = 0; p < n; ++p) out[p] = nullptr;
  if (n == 0) return PH_OK;
  cudaStream_t s = (cudaStream_t)stream;
  // host offsets: tets, Neumann triples, vertices
  std::vector<int64_t> toff(n + 1, 0), noff(n + 1, 0), voff(n + 1, 0);
  std::vector<UnionSources> src(n);
  for (int32_t p = 0; p < n; ++p) {
    const int64_t np = nN ? nN[p] : 0;
    if (nE[p] < 0 || nC[p] < 0 || np < 0 || (nE[p] > 0 && (!coord[p] || !tet[p])) ||
        (np > 0 && (!neumann || !neumann[p])) || (reinterpret_cast<uintptr_t>(tet[p]) & 15u) != 0)
      return PH_ERR_ARG;
    toff[p + 1] = toff[p] + nE[p];
    noff[p + 1] = noff[p] + np;
    voff[p + 1] = voff[p] + nC[p];
    src[p] = UnionSources{tet[p], np > 0 ? neumann[p] : nullptr};
  }
  const int64_t nEu = toff[n], nNu = noff[n], nCu = voff[n];
  if (16 * nEu + nNu >= ((int64_t)1 << 31) - 1 || nCu >= ((int64_t)1 << 31) - 1) return PH_ERR_OVERFLOW;
  // union inputs and the offset tables in one allocation
  Carve ic;
  const size_t o_coord = ic.take<double>(3 * nCu), o_tet = ic.take<int4>(nEu), o_nb = ic.take<int32_t>(3 * nNu);
  const size_t o_src = ic.take<UnionSources>(n), o_off = ic.take<int64_t>(3 * (n + 1));
  const size_t o_cnt = ic.take<long long>(3 * n);
  void* in = nullptr;
  cudaError_t e = alloc_bytes(&in, ic.bytes, s);
  if (e != cudaSuccess) return cuda_status(e, "alloc batch inputs");
  double* coord_u = Carve::at<double>(in, o_coord);
  int4* tet_u = Carve::at<int4>(in, o_tet);
  int32_t* nb_u = Carve::at<int32_t>(in, o_nb);
  UnionSources* d_src = Carve::at<UnionSources>(in, o_src);
  int64_t* d_off = Carve::at<int64_t>(in, o_off);  // toff, noff, voff
  long long* d_cnt = Carve::at<long long>(in, o_cnt);
  std::vector<int64_t> offs;
  offs.insert(offs.end(), toff.begin(), toff.end());
  offs.insert(offs.end(), noff.begin(), noff.end());
  offs.insert(offs.end(), voff.begin(), voff.end());
  for (int32_t p = 0; p < n && e == cudaSuccess; ++p)
    if (nC[p] > 0)
      e = cudaMemcpyAsync(coord_u + 3 * voff[p], coord[p], sizeof(double) * 3 * nC[p], cudaMemcpyDeviceToDevice, s);
  // pageable sources: the copies return once the data is staged
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_src, src.data(), sizeof(UnionSources) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_off, offs.data(), sizeof(int64_t) * offs.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && nEu + nNu > 0) {
    k_union_inputs<<<grid_for(nEu + nNu), kThreads, 0, s>>>(d_src, d_off, d_off + (n + 1), d_off + 2 * (n + 1), n,
                                                          nEu, nNu, tet_u, nb_u);
    e = launched();
  }
  if (e != cudaSuccess) {
    free_async(in, s);
    return cuda_status(e, "ph_mesh_create_batch inputs");
  }
  std::vector<long long> cnt(3 * (size_t)n, -1);
  BatchCounts bc{d_off, n, d_cnt, cnt.data()};
  ph_mesh* u = nullptr;
  ph_status st = mesh_build(coord_u, nCu, reinterpret_cast<const int32_t*>(tet_u), nEu, nNu > 0 ? nb_u : nullptr,
                            nNu, s, &u, &bc);
  free_async(in, s);
  if (st != PH_OK) return st;
  // per-problem face, multiplier and CSR offsets; an empty problem starts
  // where the next one does
  std::vector<int64_t> foff(n + 1, 0), moff(n + 1, 0), zoff(n + 1, 0);
  foff[n] = u->nF;
  moff[n] = u->L;
  zoff[n] = u->nnz;
  bool ordered = true;
  for (int32_t p = n - 1; p >= 0; --p) {
    const bool empty = cnt[3 * p] < 0;
    foff[p] = empty ? foff[p + 1] : cnt[3 * p];
    moff[p] = empty ? moff[p + 1] : cnt[3 * p + 1];
    zoff[p] = empty ? zoff[p + 1] : cnt[3 * p + 2];
    ordered = ordered && foff[p] <= foff[p + 1] && moff[p] <= moff[p + 1] && zoff[p] <= zoff[p + 1];
  }
  if (!ordered || foff[0] != 0 || moff[0] != 0 || zoff[0] != 0) {
    mesh_free(u, s);
    return PH_ERR_ARG;
  }
  // row pointers of the problems (L + n) and the offset tables (5 (n + 1))
  Carve xc;
  const size_t o_rp = xc.take<int32_t>(u->L + n), o_tab = xc.take<int64_t>(5 * (n + 1));
  void* extra = nullptr;
  e = alloc_bytes(&extra, xc.bytes, s);
  if (e != cudaSuccess) {
    mesh_free(u, s);
    return cuda_status(e, "alloc batch rows");
  }
  int32_t* rowptr_b = Carve::at<int32_t>(extra, o_rp);
  int64_t* tab = Carve::at<int64_t>(extra, o_tab);
  std::vector<int64_t> t5;
  for (const auto* v : {&toff, &voff, &foff, &moff, &zoff}) t5.insert(t5.end(), v->begin(), v->end());
  e = cudaMemcpyAsync(tab, t5.data(), sizeof(int64_t) * t5.size(), cudaMemcpyHostToDevice, s);
  const UnionOffsets o{tab, tab + (n + 1), tab + 2 * (n + 1), tab + 3 * (n + 1), tab + 4 * (n + 1), n};
  if (e == cudaSuccess && nEu > 0) {
    k_rebase_tets<<<grid_for(nEu), kThreads, 0, s>>>(o, nEu, u->tet, u->tface, u->tmult, u->tpos);
    e = launched();
  }
  if (e == cudaSuccess && u->nF > 0) {
    k_rebase_faces<<<grid_for(u->nF), kThreads, 0, s>>>(o, u->nF, u->face_tet, u->face_vtx, u->face_mult);
    e = launched();
  }
  if (e == cudaSuccess) {
    k_rebase_rows<<<grid_for(u->L + n), kThreads, 0, s>>>(o, u->L, u->rowptr, rowptr_b, u->rowdiag);
    e = launched();
  }
  if (e == cudaSuccess && u->nnz > 0) {
    k_rebase_cols<<<grid_for(u->nnz), kThreads, 0, s>>>(o, u->nnz, u->colind);
    e = launched();
  }
  if (e != cudaSuccess) {
    free_async(extra, s);
    mesh_free(u, s);
    return cuda_status(e, "ph_mesh_create_batch rebase");
  }
  // the views: each problem's slices of the union arrays, local ids
  ph_mesh_shared* sh = new ph_mesh_shared();
  sh->refs.store(n);
  sh->arena = u->arena;
  sh->extra = extra;
  for (int32_t p = 0; p < n; ++p) {
    ph_mesh* m = new ph_mesh();
    memset(m, 0, sizeof *m);
    const int64_t t0 = toff[p], v0 = voff[p], f0 = foff[p], m0 = moff[p], z0 = zoff[p];
    m->device = u->device;
    m->shared = sh;
    m->nE = nE[p];
    m->nC = nC[p];
    m->nF = foff[p + 1] - f0;
    m->L = moff[p + 1] - m0;
    m->nnz = zoff[p + 1] - z0;
    m->nFi = 4 * m->nE - m->nF;
    m->nFn = m->nF - m->L;
    m->nFd = m->nF - m->nFi - m->nFn;
    m->coord = u->coord + 3 * v0;
    m->tet = u->tet + t0;
    m->tface = u->tface + t0;
    m->tmult = u->tmult + t0;
    m->tpos = u->tpos + t0;
    m->trel = u->trel + t0;
    m->geo = u->geo + PH_GEO_STRIDE * t0;
    m->face_tet = u->face_tet + f0;
    m->face_vtx = u->face_vtx + 3 * f0;
    m->face_kind = u->face_kind + f0;
    m->face_mult = u->face_mult + f0;
    m->face_area = u->face_area + f0;
    m->rowptr = rowptr_b + m0 + p;
    m->colind = u->colind + z0;
    m->rowdiag = u->rowdiag + m0;
    m->status = u->status;
    out[p] = m;
  }
  delete u;  // its arena now belongs to the views
  return PH_OK;
}
