// Adjoint of the condensed path (not in the paper): the gradient of the misfit
//     J = 1/2 sum_T e_T' M(T) e_T,   e_T = U_T - U_obs,T   (M(T) of Eq. M(T))
// with respect to theta_T = log a_T.
//
// The forward system of Eq. VectorForm, K [U; Lambda] = [B; -b_D] with
// K = [[A, -C'], [-C, 0]], is symmetric, so the adjoint solves
// K [p; q] = [M e; 0].  Condensing as in the forward path,
//     H q = -sum_T P_T' C(T) A(T)^-1 r_T,        r_T = M(T) e_T,
//     p_T = A(T)^-1 (r_T + C(T)' q_T),
// with the same H, and since only A(T) = a_T K(T) + c M(T) depends on
// theta_T (dA/dtheta_T = a_T K(T)):
//     dJ/dtheta_T = -a_T p_T' K(T) U_T
//                 = -a_T / (6 |det E|) (D0 p_T)' adj(G_e) (D0 U_T),
// using K(T) = (|det E|/6) D0' G_e^-1 D0, det G_e = det(E)^2 and the vertex
// differences D0 x = (x1 - x0, x2 - x0, x3 - x0), in which constants cancel.
// In face terms, with the element factor Q' = Qf/9 stored by ph_assemble
// (rows sum to zero), r~_m = r at the vertex opposite face m, d_k = sigma_k |F_k|:
//     (C A^-1 r)_k = d_k (sum(r)/(c|T|) - 3 (Q' r~)_k),
//     p[o(i)]      = (sum(r) + sum_k d_k q_k)/(c|T|) + (Q' (9 r~ - 3 d q))_i.
#include <math.h>

#include "element.cuh"
#include "ph_internal.cuh"

using namespace ph_elem;

namespace {

constexpr int RT = 256;
constexpr int RB = 304;

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sm[RT / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = threadIdx.x < RT / 32 ? sm[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;
}

struct V4 {
  double x, y, z, w;
};

__device__ __forceinline__ V4 ld4(const double* p) {
  const double2* q = reinterpret_cast<const double2*>(p);
  const double2 a = __ldg(q), b = __ldg(q + 1);
  return V4{a.x, a.y, b.x, b.y};
}

// e = U - U_obs and r = M(T) e = |T|/20 (e + sum(e) 1), vertex order
__device__ __forceinline__ void misfit_load(const double* __restrict__ u, const double* __restrict__ u_obs, int64_t t,
                                            double adet, double e[4], double r[4]) {
  const V4 U = ld4(u + 4 * t), O = ld4(u_obs + 4 * t);
  e[0] = U.x - O.x; e[1] = U.y - O.y; e[2] = U.z - O.z; e[3] = U.w - O.w;
  const double se = (e[0] + e[1]) + (e[2] + e[3]);
  const double s20 = adet * (1.0 / 120.0);  // |T|/20
#pragma unroll
  for (int j = 0; j < 4; ++j) r[j] = s20 * (e[j] + se);
}

// J partial sums: 1/2 e' M e = 1/2 |T|/20 (e.e + (sum e)^2)
__global__ void __launch_bounds__(RT) k_misfit_partial(int64_t nE, const double* __restrict__ geo,
                                                       const double* __restrict__ u, const double* __restrict__ u_obs,
                                                       double* __restrict__ part) {
  double acc = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)RT + threadIdx.x; t < nE; t += (int64_t)RB * RT) {
    const double adet = __ldg(geo + PH_GEO_STRIDE * t + 15);
    double e[4], r[4];
    misfit_load(u, u_obs, t, adet, e, r);
    acc = fma(0.5, (e[0] * r[0] + e[1] * r[1]) + (e[2] * r[2] + e[3] * r[3]), acc);
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(RT) k_misfit_final(const double* __restrict__ part, double* __restrict__ J) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < RB; i += RT) acc += part[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) *J = acc;
}

__global__ void k_zero(double* __restrict__ x, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] = 0.0;
}

__device__ __forceinline__ void load_factor(const double* __restrict__ factor, int64_t t, double Q[10]) {
  const double2* fp = reinterpret_cast<const double2*>(factor + 10 * t);
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const double2 v = __ldg(fp + i);
    Q[2 * i] = v.x;
    Q[2 * i + 1] = v.y;
  }
}

// vertex opposite face k: o = (3, 1, 2, 0)
__device__ __forceinline__ int opp(int k) { return k == 0 ? 3 : (k == 3 ? 0 : k); }

// rhs_q[l(F_k)] += -(C A^-1 r)_k
__global__ void __launch_bounds__(128) k_adjoint_rhs(int64_t nE, const double* __restrict__ geo,
                                                     const int4* __restrict__ tface, const int4* __restrict__ tmult,
                                                     const double* __restrict__ face_area,
                                                     const double* __restrict__ factor, double six_over_c,
                                                     const double* __restrict__ u, const double* __restrict__ u_obs,
                                                     double* __restrict__ rhs_q) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nE) return;
  const double* gp = geo + PH_GEO_STRIDE * t;
  const double adet = __ldg(gp + 15), rdet = __ldg(gp + 16);
  double e[4], r[4];
  misfit_load(u, u_obs, t, adet, e, r);
  double Q[10];
  load_factor(factor, t, Q);
  const double icT = rdet * six_over_c;
  const double base = icT * ((r[0] + r[1]) + (r[2] + r[3]));
  const int4 tf = __ldg(tface + t), tm = __ldg(tmult + t);
  double rt[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) rt[m] = r[opp(m)];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int mk = comp(tm, k);
    if (mk == PH_NO_MULT) continue;
    const int F = comp(tf, k) & PH_ID_MASK;
    double qr = 0.0;
#pragma unroll
    for (int m = 0; m < 4; ++m) qr = fma(Q[ut(k, m)], rt[m], qr);
    const double w = neg_if(__ldg(face_area + F) * fma(-3.0, qr, base), comp(tf, k) < 0);  // (C A^-1 r)_k
    if (mk < 0)  // boundary face: the only contribution
      rhs_q[mk & PH_ID_MASK] = -w;
    else
      atomicAdd(rhs_q + (mk & PH_ID_MASK), -w);
  }
}

// dJ/dtheta_T = -a_T/(6|det|) (D0 p)' adj(G_e) (D0 U)
__global__ void __launch_bounds__(128) k_adjoint_grad(int64_t nE, const double* __restrict__ geo,
                                                      const int4* __restrict__ tface, const int4* __restrict__ tmult,
                                                      const double* __restrict__ face_area,
                                                      const double* __restrict__ a,
                                                      const double* __restrict__ factor, double six_over_c,
                                                      const double* __restrict__ u, const double* __restrict__ u_obs,
                                                      const double* __restrict__ q, double* __restrict__ grad) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nE) return;
  const Geo G = load_geo(geo, t);
  double e[4], r[4];
  misfit_load(u, u_obs, t, G.adet, e, r);
  double Q[10];
  load_factor(factor, t, Q);
  const int4 tf = __ldg(tface + t), tm = __ldg(tmult + t);
  double v[4];
  double sdq = 0.0;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int mm = comp(tm, m);
    double dq = 0.0;
    if (mm != PH_NO_MULT) {
      const int F = comp(tf, m) & PH_ID_MASK;
      dq = neg_if(__ldg(face_area + F), comp(tf, m) < 0) * __ldg(q + (mm & PH_ID_MASK));
    }
    sdq += dq;
    v[m] = fma(9.0, r[opp(m)], -3.0 * dq);
  }
  const double icT = G.rdet * six_over_c;
  const double base = icT * (((r[0] + r[1]) + (r[2] + r[3])) + sdq);
  double p[4];  // vertex order
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    double acc = base;
#pragma unroll
    for (int m = 0; m < 4; ++m) acc = fma(Q[ut(i, m)], v[m], acc);
    p[opp(i)] = acc;
  }
  const V4 U = ld4(u + 4 * t);
  const double du0 = U.y - U.x, du1 = U.z - U.x, du2 = U.w - U.x;
  const double dp0 = p[1] - p[0], dp1 = p[2] - p[0], dp2 = p[3] - p[0];
  // adj(G_e), symmetric
  const double A00 = fma(G.g11, G.g22, -G.g12 * G.g12);
  const double A01 = fma(G.g02, G.g12, -G.g01 * G.g22);
  const double A02 = fma(G.g01, G.g12, -G.g02 * G.g11);
  const double A11 = fma(G.g00, G.g22, -G.g02 * G.g02);
  const double A12 = fma(G.g01, G.g02, -G.g00 * G.g12);
  const double A22 = fma(G.g00, G.g11, -G.g01 * G.g01);
  const double w0 = fma(A00, du0, fma(A01, du1, A02 * du2));
  const double w1 = fma(A01, du0, fma(A11, du1, A12 * du2));
  const double w2 = fma(A02, du0, fma(A12, du1, A22 * du2));
  const double pKu = fma(dp0, w0, fma(dp1, w1, dp2 * w2));
  grad[t] = -__ldg(a + t) * (G.rdet * (1.0 / 6.0)) * pKu;
}

bool finite_pos(double x) { return x > 0.0 && x < INFINITY; }

}  // namespace

using namespace ph;

extern "C" ph_status ph_misfit(const ph_mesh* m, const double* u, const double* u_obs, double* J, void* stream) {
  if (!m || !J || (m->nE > 0 && (!u || !u_obs))) return PH_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  double* part = nullptr;
  cudaError_t e = alloc(&part, RB, s);
  if (e != cudaSuccess) return cuda_status(e, "ph_misfit alloc");
  k_misfit_partial<<<RB, RT, 0, s>>>(m->nE, m->geo, u, u_obs, part);
  k_misfit_final<<<1, RT, 0, s>>>(part, J);
  e = launched(2);
  free_async(part, s);
  return cuda_status(e, "ph_misfit");
}

extern "C" ph_status ph_adjoint_rhs(const ph_mesh* m, const double* factor, double c, const double* u,
                                    const double* u_obs, double* rhs_q, void* stream) {
  if (!m || !finite_pos(c)) return PH_ERR_ARG;
  if (m->nE > 0 && (!factor || !u || !u_obs)) return PH_ERR_ARG;
  if (m->L > 0 && !rhs_q) return PH_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (m->L > 0) {
    k_zero<<<grid_for(m->L), kThreads, 0, s>>>(rhs_q, m->L);
    cudaError_t e = launched();
    if (e != cudaSuccess) return cuda_status(e, "k_zero");
  }
  if (m->nE == 0) return PH_OK;
  k_adjoint_rhs<<<grid_for(m->nE, 128), 128, 0, s>>>(m->nE, m->geo, m->tface, m->tmult, m->face_area, factor, 6.0 / c,
                                                     u, u_obs, rhs_q);
  return cuda_status(launched(), "k_adjoint_rhs");
}

extern "C" ph_status ph_adjoint_grad(const ph_mesh* m, const double* a, const double* factor, double c,
                                     const double* u, const double* u_obs, const double* q, double* grad,
                                     void* stream) {
  if (!m || !finite_pos(c)) return PH_ERR_ARG;
  if (m->geo_dw) {  // the gradient reads G_e from the fp64 geometry record
    set_error_text("ph_adjoint_grad: the mesh holds a double-word geometry record (ph_mesh_create_dw)");
    return PH_ERR_ARG;
  }
  if (m->nE > 0 && (!a || !factor || !u || !u_obs || !grad || (m->L > 0 && !q))) return PH_ERR_ARG;
  if (m->nE == 0) return PH_OK;
  cudaStream_t s = (cudaStream_t)stream;
  k_adjoint_grad<<<grid_for(m->nE, 128), 128, 0, s>>>(m->nE, m->geo, m->tface, m->tmult, m->face_area, a, factor,
                                                      6.0 / c, u, u_obs, q, grad);
  return cuda_status(launched(), "k_adjoint_grad");
}
