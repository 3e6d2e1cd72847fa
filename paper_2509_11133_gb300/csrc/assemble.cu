// Per-element local matrices, Schur condensation onto the face multipliers and
// scatter into CSR (Section 4.2-4.3, Eq. schur, Algorithm 1 first loop), and
// element recovery (Algorithm 1 second loop).  One thread per tetrahedron.
//
// Element algebra.  With A = a K + c M (Eqs. K(T), M(T)) and the constant
// vector 1: K 1 = 0 and M 1 = |T|/4 1, and M = |T|/20 I on the complement of 1.
// Hence, exactly,
//     A^-1 = J / (c|T|) + Qv,   J = 1 1',
// where Qv is the inverse of (aK + c|T|/20 I) on the complement of 1.  Writing
// E for the 3x3 matrix with rows P_i - P_0 (i = 1..3), G_e = E E',
// T0 = I + 1 1' (3x3) and D0 = [-1 | I] (3x4), the gradients of the barycentric
// coordinates are E^-1 D0 and K = (|det E|/6) D0' E^-T E^-1 D0, which gives
//     Qv = (6/|det E|) D0' (a T0 + (c/20) G_e)^-1 G_e T0^-1 D0.
// The 3x3 matrix a T0 + (c/20) G_e has condition number ~4 for any element
// with a >> c h^2, so this form keeps full fp64 accuracy where forming A and
// solving with it loses ~log10(a/(c h^2)) digits.  Qv 1 = 0.
//
// With C(T) = diag(sigma_k |F_k|) R (Eq. C(T)) and the rows r_k = (1 - e_o(k))/3,
// o = (3, 1, 2, 0) the vertex opposite face k, and Qf[k][m] = Qv[o(k)][o(m)]:
//     S[k][m] = d_k d_m (1/(c|T|) + Qf[k][m]/9),            d_k = sigma_k |F_k|,
//     g[k]    = -d_k (h'sum/(c|T|) + (Qf h')_k / 9),
//     h'_k    = |T|/4 f(Ct_k) + |F_k| g_N(Ct_k) [k Neumann],
// (the load B_j = sum_k h'_k/3 [j != o(k)] is the paper's face-centroid rule),
// and recovery U(T) = A^-1 (B + C' Lambda_T) is
//     U[o(k)] = z'sum/(c|T|) - (Qf z')_k / 3,   z'_k = h'_k + d_k Lambda_k.
// G_e and G_e T0^-1 come precomputed per element from the mesh (they depend
// on the geometry only).  ph_assemble can also store Qf/9 per element (the
// "element factor", 10 numbers) so that ph_recover_factored skips the
// condensation kernel.
#include <math.h>
#include <stdio.h>

#include "element.cuh"
#include "ph_internal.cuh"

using namespace ph_elem;

namespace {

template <bool UD, bool GN, bool FAC, int MODE>
__global__ void __launch_bounds__(128, MODE ? 7 : 1) k_assemble(int64_t nE, const double* __restrict__ geo,
                                                  const int4* __restrict__ tface, const int4* __restrict__ tmult,
                                                  const int4* __restrict__ tpos, const ushort4* __restrict__ trel,
                                                  const double* __restrict__ face_area, const double* __restrict__ a,
                                                  double c20, double six_over_c, const double* __restrict__ f_face,
                                                  const double* __restrict__ uD, const double* __restrict__ gN,
                                                  double* __restrict__ values, double* __restrict__ rhs,
                                                  double* __restrict__ factor, unsigned* status,
                                                  const double* __restrict__ coord, const int4* __restrict__ tet) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nE) return;
  assemble_element<UD, GN, FAC, MODE>(t, geo, tface, tmult, tpos, trel, face_area, a, c20, six_over_c, f_face, uD,
                                      gN, values, rhs, factor, status, coord, tet);
}


template <bool GN>
__global__ void __launch_bounds__(128) k_recover(int64_t nE, const double* __restrict__ geo,
                                                 const int4* __restrict__ tface, const int4* __restrict__ tmult,
                                                 const double* __restrict__ face_area, const double* __restrict__ a,
                                                 double c20, double six_over_c, const double* __restrict__ f_face,
                                                 const double* __restrict__ gN, const double* __restrict__ lambda,
                                                 double* __restrict__ u, unsigned* status) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nE) return;
  const double at = __ldg(a + t);
  if (!ph::pos_finite(at)) {
    ph_flag(status, PH_ERR_ARG);
    return;
  }
  const Geo G = load_geo(geo, t);
  double z[4];
  recovery_load<GN>(G.adet * (1.0 / 24.0), __ldg(tface + t), __ldg(tmult + t), face_area, f_face, gN, lambda, z);
  double Q[10];
  face_kernel(G, at, c20, -6.0 / 3.0, Q);  // -Qf/3
  const double icT = G.rdet * six_over_c;
  const double zs = icT * ((z[0] + z[1]) + (z[2] + z[3]));
  double U[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double e = zs;
#pragma unroll
    for (int m = 0; m < 4; ++m) e = fma(Q[ut(k, m)], z[m], e);
    U[k] = e;
  }
  store_u(u, t, U);
}

// Recovery from the element factor Qf/9 stored by ph_assemble.
template <bool GN>
__global__ void __launch_bounds__(128) k_recover_factored(int64_t nE, const double* __restrict__ geo,
                                                          const int4* __restrict__ tface, const int4* __restrict__ tmult,
                                                          const double* __restrict__ face_area,
                                                          const double* __restrict__ factor, double six_over_c,
                                                          const double* __restrict__ f_face,
                                                          const double* __restrict__ gN,
                                                          const double* __restrict__ lambda, double* __restrict__ u) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nE) return;
  recover_element_factored<GN>(t, geo, tface, tmult, face_area, factor, six_over_c, f_face, gN, lambda, u);
}

bool finite_pos(double x) { return x > 0.0 && x < INFINITY; }

}  // namespace

using namespace ph;

// The fp64 entry points need the fp64 geometry record, which a mesh from
// ph_mesh_create_dw does not hold.
static bool needs_fp64_record(const ph_mesh* m, const char* who) {
  if (!m->geo_dw) return false;
  char msg[160];
  snprintf(msg, sizeof msg, "%s: the mesh holds a double-word geometry record (ph_mesh_create_dw)", who);
  set_error_text(msg);
  return true;
}

template <int MODE>
static void launch_assemble(const ph_mesh* m, unsigned grid, bool ud, bool gn, double c20, double six_over_c,
                            const double* a, const double* f_face, const double* uD_face, const double* gN_face,
                            double* values, double* rhs, double* factor, cudaStream_t s) {
#define PH_ASM(UDV, GNV, FACV)                                                                                  \
  k_assemble<UDV, GNV, FACV, MODE><<<grid, 128, 0, s>>>(m->nE, m->geo, m->tface, m->tmult, m->tpos, m->trel,   \
                                                        m->face_area, a, c20, six_over_c, f_face, uD_face,     \
                                                        gN_face, values, rhs, factor, m->status, m->coord, m->tet)
  if (factor) {
    if (ud && gn) PH_ASM(true, true, true);
    else if (ud) PH_ASM(true, false, true);
    else if (gn) PH_ASM(false, true, true);
    else PH_ASM(false, false, true);
  } else {
    if (ud && gn) PH_ASM(true, true, false);
    else if (ud) PH_ASM(true, false, false);
    else if (gn) PH_ASM(false, true, false);
    else PH_ASM(false, false, false);
  }
#undef PH_ASM
}

template <bool DW>
static ph_status assemble(const ph_mesh* m, const double* a, double c, const double* f_face, const double* uD_face,
                          const double* gN_face, double* values, double* rhs, double* factor, void* stream) {
  if (!m || !finite_pos(c)) return PH_ERR_ARG;
  if (!DW && needs_fp64_record(m, "ph_assemble")) return PH_ERR_ARG;
  if (m->nE > 0 && (!a || !f_face)) return PH_ERR_ARG;
  if ((m->nnz > 0 && !values) || (m->L > 0 && !rhs)) return PH_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // The diagonal and rhs entries receive two atomic contributions and must
  // start at zero.  Clearing the whole arrays writes full 32-byte sectors
  // (faster than 8-byte scattered stores to the diagonal positions, which make
  // L2 read each sector first); the off-diagonal entries are overwritten.
  if (m->L > 0) {
    KernelTimer kt("zero_values", s);
    cudaError_t e = cudaMemsetAsync(values, 0, sizeof(double) * m->nnz, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(rhs, 0, sizeof(double) * m->L, s);
    kt.stop();
    if (e != cudaSuccess) return cuda_status(e, "zero values");
  }
  if (m->nE == 0) return PH_OK;
  const double c20 = c / 20.0, six_over_c = 6.0 / c;
  const unsigned grid = grid_for(m->nE, 128);
  const bool ud = uD_face != nullptr && m->nFd > 0, gn = gN_face != nullptr && m->nFn > 0;
  KernelTimer kt(DW ? "k_assemble_dw" : "k_assemble", s);
  if (!DW)
    launch_assemble<0>(m, grid, ud, gn, c20, six_over_c, a, f_face, uD_face, gN_face, values, rhs, factor, s);
  else if (!m->geo_dw)
    launch_assemble<1>(m, grid, ud, gn, c20, six_over_c, a, f_face, uD_face, gN_face, values, rhs, factor, s);
  else
    launch_assemble<2>(m, grid, ud, gn, c20, six_over_c, a, f_face, uD_face, gN_face, values, rhs, factor, s);
  const cudaError_t e = launched();
  kt.stop();
  return cuda_status(e, "k_assemble");
}

extern "C" ph_status ph_assemble(const ph_mesh* m, const double* a, double c, const double* f_face,
                                 const double* uD_face, const double* gN_face, double* values, double* rhs,
                                 double* factor, void* stream) {
  return assemble<false>(m, a, c, f_face, uD_face, gN_face, values, rhs, factor, stream);
}

template <bool GN>
__global__ void __launch_bounds__(128) k_recover_factored_dw(int64_t nE, const double* __restrict__ geo,
                                                             const int4* __restrict__ tface,
                                                             const int4* __restrict__ tmult,
                                                             const double* __restrict__ face_area,
                                                             const double* __restrict__ factor, double six_over_c,
                                                             const double* __restrict__ f_face,
                                                             const double* __restrict__ gN,
                                                             const double* __restrict__ lambda,
                                                             double* __restrict__ u) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nE) return;
  recover_element_factored_dw<GN>(t, geo, tface, tmult, face_area, factor, six_over_c, f_face, gN, lambda, u);
}

extern "C" ph_status ph_assemble_dw(const ph_mesh* m, const double* a, double c, const double* f_face,
                                    const double* uD_face, const double* gN_face, double* values, double* rhs,
                                    double* factor, void* stream) {
  return assemble<true>(m, a, c, f_face, uD_face, gN_face, values, rhs, factor, stream);
}

extern "C" ph_status ph_recover(const ph_mesh* m, const double* a, double c, const double* f_face,
                                const double* gN_face, const double* lambda, double* u, void* stream) {
  if (!m || !finite_pos(c)) return PH_ERR_ARG;
  if (needs_fp64_record(m, "ph_recover")) return PH_ERR_ARG;
  if (m->nE > 0 && (!a || !f_face || !u || (m->L > 0 && !lambda))) return PH_ERR_ARG;
  if (m->nE == 0) return PH_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const double c20 = c / 20.0, six_over_c = 6.0 / c;
  const unsigned grid = grid_for(m->nE, 128);
  KernelTimer kt("k_recover", s);
  if (gN_face != nullptr && m->nFn > 0)
    k_recover<true><<<grid, 128, 0, s>>>(m->nE, m->geo, m->tface, m->tmult, m->face_area, a, c20, six_over_c, f_face,
                                         gN_face, lambda, u, m->status);
  else
    k_recover<false><<<grid, 128, 0, s>>>(m->nE, m->geo, m->tface, m->tmult, m->face_area, a, c20, six_over_c,
                                          f_face, gN_face, lambda, u, m->status);
  const cudaError_t e = launched();
  kt.stop();
  return cuda_status(e, "k_recover");
}

extern "C" ph_status ph_recover_factored(const ph_mesh* m, const double* factor, double c, const double* f_face,
                                         const double* gN_face, const double* lambda, double* u, void* stream) {
  if (!m || !finite_pos(c)) return PH_ERR_ARG;
  if (m->nE > 0 && (!factor || !f_face || !u || (m->L > 0 && !lambda))) return PH_ERR_ARG;
  if (m->nE == 0) return PH_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const double six_over_c = 6.0 / c;
  const unsigned grid = grid_for(m->nE, 128);
  KernelTimer kt("k_recover_factored", s);
  if (gN_face != nullptr && m->nFn > 0)
    k_recover_factored<true><<<grid, 128, 0, s>>>(m->nE, m->geo, m->tface, m->tmult, m->face_area, factor,
                                                  six_over_c, f_face, gN_face, lambda, u);
  else
    k_recover_factored<false><<<grid, 128, 0, s>>>(m->nE, m->geo, m->tface, m->tmult, m->face_area, factor,
                                                   six_over_c, f_face, gN_face, lambda, u);
  const cudaError_t e = launched();
  kt.stop();
  return cuda_status(e, "k_recover_factored");
}

extern "C" ph_status ph_recover_factored_dw(const ph_mesh* m, const double* factor, double c, const double* f_face,
                                            const double* gN_face, const double* lambda, double* u, void* stream) {
  if (!m || !finite_pos(c)) return PH_ERR_ARG;
  if (m->nE > 0 && (!factor || !f_face || !u || (m->L > 0 && !lambda))) return PH_ERR_ARG;
  if (m->nE == 0) return PH_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const double six_over_c = 6.0 / c;
  const unsigned grid = grid_for(m->nE, 128);
  KernelTimer kt("k_recover_factored_dw", s);
  if (gN_face != nullptr && m->nFn > 0)
    k_recover_factored_dw<true><<<grid, 128, 0, s>>>(m->nE, m->geo, m->tface, m->tmult, m->face_area, factor,
                                                     six_over_c, f_face, gN_face, lambda, u);
  else
    k_recover_factored_dw<false><<<grid, 128, 0, s>>>(m->nE, m->geo, m->tface, m->tmult, m->face_area, factor,
                                                      six_over_c, f_face, gN_face, lambda, u);
  const cudaError_t e = launched();
  kt.stop();
  return cuda_status(e, "k_recover_factored_dw");
}
