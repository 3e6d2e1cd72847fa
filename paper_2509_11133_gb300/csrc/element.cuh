// Per-element helpers shared by the assembly, recovery and adjoint kernels:
// the geometry record of the mesh and the condensation kernel Qf of one
// element (see assemble.cu for the derivation).
#pragma once

#include "dw.cuh"
#include "ph_internal.cuh"

namespace ph_elem {

__device__ __forceinline__ int comp(int4 v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
__device__ __forceinline__ unsigned short comps(ushort4 v, int k) {
  return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
}

// Index of (k, m), k <= m, in the packed upper triangle 00 01 02 03 11 12 13 22 23 33.
__host__ __device__ constexpr int ut(int k, int m) {
  return k <= m ? (k * 7 - k * k) / 2 + m : (m * 7 - m * m) / 2 + k;
}

struct Geo {
  double g00, g01, g02, g11, g12, g22;  // G_e
  double t00, t01, t02, t10, t11, t12, t20, t21, t22;  // G_e T0^-1
  double adet, rdet;
};

// Element geometry of tet [P0 P1 P2 P3] in fp64: E = rows P_i - P_0
// (i = 1..3), G_e = E E', GT = G_e T0^-1 = G_e - (G_e 1) 1'/4 (T0 = I + 1 1';
// one fma per entry, the quarter being exact), |det E| and 1/|det E| (the
// Newton reciprocal).  The mesh build stores it as the element's fp64
// record; the double-word kernels recompute it for elements they hand to the
// fp64 path.
__device__ __forceinline__ Geo compute_geo(const double* __restrict__ coord, int4 v) {
  const double* p0 = coord + 3 * (int64_t)v.x;
  const double* p1 = coord + 3 * (int64_t)v.y;
  const double* p2 = coord + 3 * (int64_t)v.z;
  const double* p3 = coord + 3 * (int64_t)v.w;
  const double e1x = p1[0] - p0[0], e1y = p1[1] - p0[1], e1z = p1[2] - p0[2];
  const double e2x = p2[0] - p0[0], e2y = p2[1] - p0[1], e2z = p2[2] - p0[2];
  const double e3x = p3[0] - p0[0], e3y = p3[1] - p0[1], e3z = p3[2] - p0[2];
  const double det = e1x * (e2y * e3z - e2z * e3y) + e1y * (e2z * e3x - e2x * e3z) + e1z * (e2x * e3y - e2y * e3x);
  Geo G;
  G.adet = ph::neg_if(det, __double2hiint(det) < 0);  // |det| on the sign bit
  G.g00 = e1x * e1x + e1y * e1y + e1z * e1z;
  G.g01 = e1x * e2x + e1y * e2y + e1z * e2z;
  G.g02 = e1x * e3x + e1y * e3y + e1z * e3z;
  G.g11 = e2x * e2x + e2y * e2y + e2z * e2z;
  G.g12 = e2x * e3x + e2y * e3y + e2z * e3z;
  G.g22 = e3x * e3x + e3y * e3y + e3z * e3z;
  const double r0 = (G.g00 + G.g01) + G.g02, r1 = (G.g01 + G.g11) + G.g12, r2 = (G.g02 + G.g12) + G.g22;
  G.t00 = fma(-0.25, r0, G.g00);
  G.t01 = fma(-0.25, r0, G.g01);
  G.t02 = fma(-0.25, r0, G.g02);
  G.t10 = fma(-0.25, r1, G.g01);
  G.t11 = fma(-0.25, r1, G.g11);
  G.t12 = fma(-0.25, r1, G.g12);
  G.t20 = fma(-0.25, r2, G.g02);
  G.t21 = fma(-0.25, r2, G.g12);
  G.t22 = fma(-0.25, r2, G.g22);
  G.rdet = ph::rcp_newton(G.adet);
  return G;
}

__device__ __forceinline__ Geo load_geo(const double* __restrict__ geo, int64_t t) {
  const double2* p = reinterpret_cast<const double2*>(geo + PH_GEO_STRIDE * t);
  const double2 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2), d = __ldg(p + 3), e = __ldg(p + 4);
  const double2 f = __ldg(p + 5), g = __ldg(p + 6), h = __ldg(p + 7), i = __ldg(p + 8);
  return Geo{a.x, a.y, b.x, b.y, c.x, c.y, d.x, d.y, e.x, e.y, f.x, f.y, g.x, g.y, h.x, h.y, i.x};
}

// Qf (face-indexed, packed upper triangle) times sc = sc6/6.
__device__ __forceinline__ void face_kernel(const Geo& G, double a, double c20, double sc6, double Q[10]) {
  const double a2 = a + a;
  const double m00 = fma(c20, G.g00, a2), m11 = fma(c20, G.g11, a2), m22 = fma(c20, G.g22, a2);
  const double m01 = fma(c20, G.g01, a), m02 = fma(c20, G.g02, a), m12 = fma(c20, G.g12, a);
  double A00 = fma(m11, m22, -m12 * m12);
  double A01 = fma(m02, m12, -m01 * m22);
  double A02 = fma(m01, m12, -m02 * m11);
  double A11 = fma(m00, m22, -m02 * m02);
  double A12 = fma(m01, m02, -m00 * m12);
  double A22 = fma(m00, m11, -m01 * m01);
  const double detM = fma(m00, A00, fma(m01, A01, m02 * A02));
  const double s = (sc6 * G.rdet) * ph::rcp_newton(detM);  // sc * 6/|det E| / det M
  A00 *= s; A01 *= s; A02 *= s; A11 *= s; A12 *= s; A22 *= s;
  // Y = adj(M) G_e T0^-1 (symmetric): upper triangle
  const double y00 = fma(A00, G.t00, fma(A01, G.t10, A02 * G.t20));
  const double y01 = fma(A00, G.t01, fma(A01, G.t11, A02 * G.t21));
  const double y02 = fma(A00, G.t02, fma(A01, G.t12, A02 * G.t22));
  const double y11 = fma(A01, G.t01, fma(A11, G.t11, A12 * G.t21));
  const double y12 = fma(A01, G.t02, fma(A11, G.t12, A12 * G.t22));
  const double y22 = fma(A02, G.t02, fma(A12, G.t12, A22 * G.t22));
  // Qv = D0' Y D0; faces 0,1,2,3 sit opposite vertices 3,1,2,0
  const double c0 = y00 + y01 + y02, c1 = y01 + y11 + y12, c2 = y02 + y12 + y22;
  Q[ut(0, 0)] = y22;
  Q[ut(0, 1)] = y02;
  Q[ut(0, 2)] = y12;
  Q[ut(0, 3)] = ph::negate(c2);
  Q[ut(1, 1)] = y00;
  Q[ut(1, 2)] = y01;
  Q[ut(1, 3)] = ph::negate(c0);
  Q[ut(2, 2)] = y11;
  Q[ut(2, 3)] = ph::negate(c1);
  Q[ut(3, 3)] = c0 + c1 + c2;
}

// The geometry of one element in double-word form: G' = 2^-kg G_e and
// G'T = 2^-kg G_e T0^-1, 2^kg the binade of the largest diagonal entry of
// G_e (so every value is below ~8 in magnitude), |det E| and 1/|det E| in
// fp64, and the binade of |det E|^2 / (g00 g11 g22) (the element's
// flatness, within a factor 16).
struct GeoDW {
  dw::f2 g[6];  // G' 00 01 02 11 12 22
  dw::f2 t[9];  // G'T row-major
  double adet, rdet;
  int kg, flat;
};

// The double-word geometry from the fp64 record (integer conversions).
__device__ __forceinline__ GeoDW geo_dw_from(const Geo& G) {
  using namespace dw;
  GeoDW D;
  const int e0 = exponent(G.g00), e1 = exponent(G.g11), e2 = exponent(G.g22);
  D.kg = max(e0, max(e1, e2));
  D.flat = -2 * exponent(G.rdet) - (e0 + e1 + e2);
  const int s = -D.kg;
  D.g[0] = from_double(G.g00, s);
  D.g[1] = from_double(G.g01, s);
  D.g[2] = from_double(G.g02, s);
  D.g[3] = from_double(G.g11, s);
  D.g[4] = from_double(G.g12, s);
  D.g[5] = from_double(G.g22, s);
  D.t[0] = from_double(G.t00, s);
  D.t[1] = from_double(G.t01, s);
  D.t[2] = from_double(G.t02, s);
  D.t[3] = from_double(G.t10, s);
  D.t[4] = from_double(G.t11, s);
  D.t[5] = from_double(G.t12, s);
  D.t[6] = from_double(G.t20, s);
  D.t[7] = from_double(G.t21, s);
  D.t[8] = from_double(G.t22, s);
  D.adet = G.adet;
  D.rdet = G.rdet;
  return D;
}

// The double-word record of a mesh built by ph_mesh_create_dw (same 144 bytes
// per element as the fp64 record: 30 floats of pairs, then |det E| and
// 1/|det E| as doubles 15 and 16, then kg and the flatness as two ints).
__device__ __forceinline__ GeoDW load_geo_dw(const double* __restrict__ geo, int64_t t) {
  const float4* p = reinterpret_cast<const float4*>(geo + PH_GEO_STRIDE * t);
  float v[36];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const float4 q = __ldg(p + i);
    v[4 * i] = q.x;
    v[4 * i + 1] = q.y;
    v[4 * i + 2] = q.z;
    v[4 * i + 3] = q.w;
  }
  GeoDW D;
#pragma unroll
  for (int i = 0; i < 6; ++i) D.g[i] = dw::f2{v[2 * i], v[2 * i + 1]};
#pragma unroll
  for (int i = 0; i < 9; ++i) D.t[i] = dw::f2{v[12 + 2 * i], v[13 + 2 * i]};
  D.adet = __hiloint2double(__float_as_int(v[31]), __float_as_int(v[30]));
  D.rdet = __hiloint2double(__float_as_int(v[33]), __float_as_int(v[32]));
  D.kg = __float_as_int(v[34]);
  D.flat = __float_as_int(v[35]);
  return D;
}

// The same Qf (times sc = sc6/6) with the 3x3 algebra in double-word
// arithmetic on the FP32 pipe (dw.cuh), for the assembly variant of
// ph_assemble_dw.  The element is first made dimensionless with exact powers
// of two: G_e and G_e T0^-1 are scaled by 2^-k, 2^k the largest diagonal
// entry's binade, so that
//     Qv = 6 / (a |det E|) 2^k D0' (T0 + gamma G')^-1 G'T D0,
//     G' = 2^-k G_e, G'T = 2^-k G_e T0^-1, gamma = c 2^k / (20 a),
// and the double-word values stay within a few binades of 1; the scalar's
// power of two goes into the conversion back to fp64.  The path is taken when
// gamma G' is small against T0 (gamma 2^-k max g_ii <= 2^-2: the 3x3 matrix
// then has condition number <= 6 and the double-word result is accurate to
// ~1e-14 relative) and the element is not flat (|det E|^2 >= 2^-12 g00 g11
// g22, judged on the exponents: the Kuhn elements and their refinements
// sit near 2^-3, the jittered ones above 2^-10; on flatter elements the
// condensation kernel's cancellations would cost the float pairs' 5 bits
// fewer than fp64 more than the 1e-12 the results are held to).  Otherwise
// -- a reaction term that dominates the element (c h^2 > a), a flat element,
// or inputs beyond the exponent range -- it returns false and the caller
// takes the fp64 path.
__device__ __forceinline__ bool face_kernel_dw(const GeoDW& D, double a, double c20, double sc6, double Q[10]) {
  using namespace dw;
  const int kg = D.kg;
  const int ka = exponent(a), kc = exponent(c20), kr = exponent(D.rdet);
  const int p = kc + kg - ka;  // binade of gamma (within a factor 4)
  const int K = kr - ka + kg;  // binade of the overall scalar 6/(a |det E|) 2^k (with sc)
  if (p > -4 || D.flat < -12 || kg < -900 || kg > 900 || ka < -900 || ka > 900 || K < -900 || K > 900) return false;
  const f2 am = from_double(a, -ka), cm = from_double(c20, -kc);  // mantissas in [1, 2)
  const f2 ra = rcp(am);
  // gamma G' and the 3x3 matrix T0 + gamma G' (T0 = I + 1 1')
  f2 m00, m01, m02, m11, m12, m22;
  if (p < -100) {  // gamma G' below 2^-98 of T0: T0 alone
    m00 = m11 = m22 = f2{2.f, 0.f};
    m01 = m02 = m12 = f2{1.f, 0.f};
  } else {
    const f2 gam = ldexp(mul(cm, ra), p);
    m00 = add(mul(gam, D.g[0]), 2.f);
    m01 = add(mul(gam, D.g[1]), 1.f);
    m02 = add(mul(gam, D.g[2]), 1.f);
    m11 = add(mul(gam, D.g[3]), 2.f);
    m12 = add(mul(gam, D.g[4]), 1.f);
    m22 = add(mul(gam, D.g[5]), 2.f);
  }
  // adjugate and determinant
  const f2 A00 = sub(mul(m11, m22), mul(m12, m12));
  const f2 A01 = sub(mul(m02, m12), mul(m01, m22));
  const f2 A02 = sub(mul(m01, m12), mul(m02, m11));
  const f2 A11 = sub(mul(m00, m22), mul(m02, m02));
  const f2 A12 = sub(mul(m01, m02), mul(m00, m12));
  const f2 A22 = sub(mul(m00, m11), mul(m01, m01));
  const f2 det = add(add(mul(m00, A00), mul(m01, A01)), mul(m02, A02));
  // scalar: sc 6/(a |det E|) / det M' with its power of two 2^K kept apart
  const f2 sc = mul(mul(mul(from_double(sc6), from_double(D.rdet, -kr)), ra), rcp(det));
  const f2* t = D.t;
  // Y = adj(M') G'T (symmetric), scaled
  const f2 y00 = mul(add(add(mul(A00, t[0]), mul(A01, t[3])), mul(A02, t[6])), sc);
  const f2 y01 = mul(add(add(mul(A00, t[1]), mul(A01, t[4])), mul(A02, t[7])), sc);
  const f2 y02 = mul(add(add(mul(A00, t[2]), mul(A01, t[5])), mul(A02, t[8])), sc);
  const f2 y11 = mul(add(add(mul(A01, t[1]), mul(A11, t[4])), mul(A12, t[7])), sc);
  const f2 y12 = mul(add(add(mul(A01, t[2]), mul(A11, t[5])), mul(A12, t[8])), sc);
  const f2 y22 = mul(add(add(mul(A02, t[2]), mul(A12, t[5])), mul(A22, t[8])), sc);
  // Qv = D0' Y D0; faces 0,1,2,3 sit opposite vertices 3,1,2,0
  const f2 c0 = add(add(y00, y01), y02), c1 = add(add(y01, y11), y12), c2 = add(add(y02, y12), y22);
  Q[ut(0, 0)] = to_double(y22, K);
  Q[ut(0, 1)] = to_double(y02, K);
  Q[ut(0, 2)] = to_double(y12, K);
  Q[ut(0, 3)] = to_double(neg(c2), K);
  Q[ut(1, 1)] = to_double(y00, K);
  Q[ut(1, 2)] = to_double(y01, K);
  Q[ut(1, 3)] = to_double(neg(c0), K);
  Q[ut(2, 2)] = to_double(y11, K);
  Q[ut(2, 3)] = to_double(neg(c1), K);
  Q[ut(3, 3)] = to_double(add(add(c0, c1), c2), K);
  return true;
}

using ph::neg_if;


// Local matrices, condensation and scatter of element t (Section 4.2-4.3,
// Eq. schur): the body of the assembly kernels (one thread per element).
// MODE: 0 fp64 (the fp64 record, face_kernel); 1 the double-word face
// kernel on the fp64 record (converted); 2 the double-word record of a mesh
// from ph_mesh_create_dw (elements the double-word kernel hands back get
// their fp64 geometry recomputed from coord and tet).
template <bool UD, bool GN, bool FAC, int MODE = 0>
__device__ __forceinline__ void assemble_element(int64_t t, const double* __restrict__ geo,
                                                 const int4* __restrict__ tface, const int4* __restrict__ tmult,
                                                 const int4* __restrict__ tpos, const ushort4* __restrict__ trel,
                                                 const double* __restrict__ face_area, const double* __restrict__ a,
                                                 double c20, double six_over_c, const double* __restrict__ f_face,
                                                 const double* __restrict__ uD, const double* __restrict__ gN,
                                                 double* __restrict__ values, double* __restrict__ rhs,
                                                 double* __restrict__ factor, unsigned* status,
                                                 const double* __restrict__ coord = nullptr,
                                                 const int4* __restrict__ tet = nullptr) {
  const double at = __ldg(a + t);
  if (!ph::pos_finite(at)) {
    ph_flag(status, PH_ERR_ARG);
    return;
  }
  Geo G;
  GeoDW D;
  if (MODE == 2) {
    D = load_geo_dw(geo, t);
    G.adet = D.adet;
    G.rdet = D.rdet;
  } else {
    G = load_geo(geo, t);
    if (MODE == 1) D = geo_dw_from(G);
  }
  const int4 tf = __ldg(tface + t);
  const int4 tm = __ldg(tmult + t);
  int F[4];
  bool neg[4];
  double ar[4], h[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    F[k] = comp(tf, k) & PH_ID_MASK;
    neg[k] = comp(tf, k) < 0;
    ar[k] = __ldg(face_area + F[k]);
  }
  const double q4 = G.adet * (1.0 / 24.0);  // |T| / 4
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    h[k] = q4 * __ldg(f_face + F[k]);
    if (GN && comp(tm, k) == PH_NO_MULT) h[k] = fma(ar[k], __ldg(gN + F[k]), h[k]);
  }
  double Q[10];
  if (MODE == 0) {
    face_kernel(G, at, c20, 6.0 / 9.0, Q);
  } else if (!face_kernel_dw(D, at, c20, 6.0 / 9.0, Q)) {
    if (MODE == 2) G = compute_geo(coord, __ldg(tet + t));
    face_kernel(G, at, c20, 6.0 / 9.0, Q);
  }
  if (FAC) {
    double2* fo = reinterpret_cast<double2*>(factor + 10 * t);
    fo[0] = make_double2(Q[0], Q[1]);
    fo[1] = make_double2(Q[2], Q[3]);
    fo[2] = make_double2(Q[4], Q[5]);
    fo[3] = make_double2(Q[6], Q[7]);
    fo[4] = make_double2(Q[8], Q[9]);
  }
  const double icT = G.rdet * six_over_c;  // 1/(c|T|)
  const double hs = (h[0] + h[1]) + (h[2] + h[3]);
  const double base = icT * hs;
  // condensed block S[k][m] = d_k d_m (1/(c|T|) + Qf/9), each entry once, as
  // d_k (Q_km d_m + e_m) with d = sigma |F| (sign on the bit pattern) and
  // e_m = d_m / (c|T|): 4 + 2 per entry FP64 operations
  double d[4], e4[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    d[k] = neg_if(ar[k], neg[k]);
    e4[k] = icT * d[k];
  }
  double S[10];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int m = k; m < 4; ++m) S[ut(k, m)] = d[k] * fma(Q[ut(k, m)], d[m], e4[m]);
  const int4 tp = __ldg(tpos + t);
  const ushort4 tr = __ldg(trel + t);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int mk = comp(tm, k);
    if (mk == PH_NO_MULT) continue;
    const int l = mk & PH_ID_MASK;
    const bool bnd = mk < 0;
    // g_k = -d_k (h'sum/(c|T|) + (Qf h')_k / 9)
    double e = base;
#pragma unroll
    for (int m = 0; m < 4; ++m) e = fma(Q[ut(k, m)], h[m], e);
    double g = neg_if(ar[k] * e, !neg[k]);
    if (UD && bnd) g = fma(ar[k], __ldg(uD + F[k]), g);  // b_D = |F| u_D(Ct_F)
    const int pd = comp(tp, k);
    if (bnd) {
      values[pd] = S[ut(k, k)];
      rhs[l] = g;
    } else {
      atomicAdd(values + pd, S[ut(k, k)]);
      atomicAdd(rhs + l, g);
    }
    const unsigned rel = comps(tr, k);
    int idx = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      if (m == k) continue;
      if (comp(tm, m) != PH_NO_MULT) {
        const int off = ((int)(rel << (28 - 4 * idx))) >> 28;  // sign-extend 4 bits
        values[pd + off] = S[ut(k, m)];
      }
      ++idx;
    }
  }
}

__device__ __forceinline__ void store_u(double* __restrict__ u, int64_t t, const double U[4]) {
  // vertex j holds U of the face opposite it: j = 0,1,2,3 <- k = 3,1,2,0
  double2* out = reinterpret_cast<double2*>(u + 4 * t);
  out[0] = make_double2(U[3], U[1]);
  out[1] = make_double2(U[2], U[0]);
}

// z'_k = |T|/4 f(Ct_k) + |F_k| g(Ct_k) [Neumann] + d_k Lambda_k
template <bool GN>
__device__ __forceinline__ void recovery_load(double q4, int4 tf, int4 tm, const double* __restrict__ face_area,
                                              const double* __restrict__ f_face, const double* __restrict__ gN,
                                              const double* __restrict__ lambda, double z[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int F = comp(tf, k) & PH_ID_MASK;
    const int mk = comp(tm, k);
    const double ar = __ldg(face_area + F);
    double zk = q4 * __ldg(f_face + F);
    if (mk == PH_NO_MULT) {
      if (GN) zk = fma(ar, __ldg(gN + F), zk);
    } else {
      zk = fma(neg_if(ar, comp(tf, k) < 0), __ldg(lambda + (mk & PH_ID_MASK)), zk);
    }
    z[k] = zk;
  }
}

// Recovery of element t from the element factor Qf/9 stored by the assembly
// (Algorithm 1, second loop): U[o(k)] = z'sum/(c|T|) - 3 (Qf/9 z')_k.  The
// body of the plain and the batched recovery kernels.
template <bool GN>
__device__ __forceinline__ void recover_element_factored(int64_t t, const double* __restrict__ geo,
                                                         const int4* __restrict__ tface,
                                                         const int4* __restrict__ tmult,
                                                         const double* __restrict__ face_area,
                                                         const double* __restrict__ factor, double six_over_c,
                                                         const double* __restrict__ f_face,
                                                         const double* __restrict__ gN,
                                                         const double* __restrict__ lambda, double* __restrict__ u) {
  const double2 dr = __ldg(reinterpret_cast<const double2*>(geo + PH_GEO_STRIDE * t) + 7);  // (t22, |det|)
  const double rdet = __ldg(geo + PH_GEO_STRIDE * t + 16);
  double z[4];
  recovery_load<GN>(dr.y * (1.0 / 24.0), __ldg(tface + t), __ldg(tmult + t), face_area, f_face, gN, lambda, z);
  const double2* fp = reinterpret_cast<const double2*>(factor + 10 * t);
  const double2 q0 = __ldg(fp), q1 = __ldg(fp + 1), q2 = __ldg(fp + 2), q3 = __ldg(fp + 3), q4 = __ldg(fp + 4);
  const double Q[10] = {q0.x, q0.y, q1.x, q1.y, q2.x, q2.y, q3.x, q3.y, q4.x, q4.y};
  const double icT = rdet * six_over_c;
  const double zs = icT * ((z[0] + z[1]) + (z[2] + z[3]));
  double U[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double e = 0.0;
#pragma unroll
    for (int m = 0; m < 4; ++m) e = fma(Q[ut(k, m)], z[m], e);
    U[k] = fma(-3.0, e, zs);
  }
  store_u(u, t, U);
}

// The same recovery with the product (Qf/9) z' in double-word arithmetic on
// the FP32 pipe (dw.cuh): the factor and z' become float pairs scaled by the
// element's largest binade of each, each row sum returns to fp64 exactly
// scaled.  z', its sum and the final combination stay fp64: they are the
// terms whose rounding bounds the result when a Lambda that is not a
// solution makes them cancel, and the pairs' ~2^-47 lands on the smaller
// (Qf z')/3 (a factor c h^2/a below them).  18 FP64 operations per element
// instead of 34.  Elements whose binades leave the pairs' range take the fp64
// product.
template <bool GN>
__device__ __forceinline__ void recover_element_factored_dw(int64_t t, const double* __restrict__ geo,
                                                            const int4* __restrict__ tface,
                                                            const int4* __restrict__ tmult,
                                                            const double* __restrict__ face_area,
                                                            const double* __restrict__ factor, double six_over_c,
                                                            const double* __restrict__ f_face,
                                                            const double* __restrict__ gN,
                                                            const double* __restrict__ lambda,
                                                            double* __restrict__ u) {
  using namespace dw;
  const double2 dr = __ldg(reinterpret_cast<const double2*>(geo + PH_GEO_STRIDE * t) + 7);  // (t22, |det|)
  const double rdet = __ldg(geo + PH_GEO_STRIDE * t + 16);
  double z[4];
  recovery_load<GN>(dr.y * (1.0 / 24.0), __ldg(tface + t), __ldg(tmult + t), face_area, f_face, gN, lambda, z);
  const double2* fp = reinterpret_cast<const double2*>(factor + 10 * t);
  const double2 q0 = __ldg(fp), q1 = __ldg(fp + 1), q2 = __ldg(fp + 2), q3 = __ldg(fp + 3), q4 = __ldg(fp + 4);
  const double Q[10] = {q0.x, q0.y, q1.x, q1.y, q2.x, q2.y, q3.x, q3.y, q4.x, q4.y};
  const double icT = rdet * six_over_c;
  const double zs = icT * ((z[0] + z[1]) + (z[2] + z[3]));
  int kq = -1023, kz = -1023;
#pragma unroll
  for (int i = 0; i < 10; ++i) kq = max(kq, exponent(Q[i]));
#pragma unroll
  for (int m = 0; m < 4; ++m) kz = max(kz, exponent(z[m]));
  double U[4];
  if (kq > -900 && kq < 900 && kz > -900 && kz < 900 && kq + kz > -1000 && kq + kz < 1000) {
    f2 qd[10], zd[4];
#pragma unroll
    for (int i = 0; i < 10; ++i) qd[i] = from_double(Q[i], -kq);
#pragma unroll
    for (int m = 0; m < 4; ++m) zd[m] = from_double(z[m], -kz);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      f2 v = mul(qd[ut(k, 0)], zd[0]);
#pragma unroll
      for (int m = 1; m < 4; ++m) v = add(v, mul(qd[ut(k, m)], zd[m]));
      U[k] = fma(-3.0, to_double(v, kq + kz), zs);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double e = 0.0;
#pragma unroll
      for (int m = 0; m < 4; ++m) e = fma(Q[ut(k, m)], z[m], e);
      U[k] = fma(-3.0, e, zs);
    }
  }
  store_u(u, t, U);
}

}  // namespace ph_elem
