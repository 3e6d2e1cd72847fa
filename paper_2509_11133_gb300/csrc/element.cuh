// Per-element helpers shared by the assembly, recovery and adjoint kernels:
// the geometry record of the mesh and the condensation kernel Qf of one
// element (see assemble.cu for the derivation).
#pragma once

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

using ph::neg_if;


// Local matrices, condensation and scatter of element t (Section 4.2-4.3,
// Eq. schur): the body of the assembly kernels (one thread per element).
template <bool UD, bool GN, bool FAC>
__device__ __forceinline__ void assemble_element(int64_t t, const double* __restrict__ geo,
                                                 const int4* __restrict__ tface, const int4* __restrict__ tmult,
                                                 const int4* __restrict__ tpos, const ushort4* __restrict__ trel,
                                                 const double* __restrict__ face_area, const double* __restrict__ a,
                                                 double c20, double six_over_c, const double* __restrict__ f_face,
                                                 const double* __restrict__ uD, const double* __restrict__ gN,
                                                 double* __restrict__ values, double* __restrict__ rhs,
                                                 double* __restrict__ factor, unsigned* status) {
  const double at = __ldg(a + t);
  if (!ph::pos_finite(at)) {
    ph_flag(status, PH_ERR_ARG);
    return;
  }
  const Geo G = load_geo(geo, t);
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
  face_kernel(G, at, c20, 6.0 / 9.0, Q);
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

}  // namespace ph_elem
