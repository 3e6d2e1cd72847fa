// Jacobi-preconditioned conjugate gradients for the condensed face system
// H Lambda = rhs (Eq. schur; the paper solves it with MATLAB's backslash).
// All reductions use a fixed grid and a fixed summation order, so repeated
// solves are bitwise reproducible.
#include <math.h>

#include "pcg.cuh"
#include "ph_internal.cuh"

namespace {

using namespace ph_pcg;

// Workspace of one solve (doubles): r, p, q, dinv (4 vectors of vec_stride(n)
// doubles, so each starts 256-byte aligned), then the partial sums, then
// Scalars.
inline size_t vec_stride(int64_t n) { return ((size_t)n + 31) & ~(size_t)31; }
inline size_t workspace_doubles(int64_t n) { return 4 * vec_stride(n) + kPart + (sizeof(Scalars) + 7) / 8; }

__global__ void __launch_bounds__(RT) k_pcg_init(int64_t n, const int32_t* __restrict__ rowptr,
                                                 const int32_t* __restrict__ colind, const double* __restrict__ val,
                                                 const double* __restrict__ b, double* __restrict__ x,
                                                 double* __restrict__ r, double* __restrict__ p,
                                                 double* __restrict__ dinv, double* __restrict__ part,
                                                 Scalars* __restrict__ sc) {
  double rz = 0.0, bb = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)RB * RT) {
    double d = 0.0;
    for (int j = rowptr[i]; j < rowptr[i + 1]; ++j)
      if (colind[j] == i) d = val[j];
    if (!(d > 0.0)) atomicOr(&sc->bad, 1u);
    const double di = d > 0.0 ? 1.0 / d : 0.0;
    const double bi = b[i];
    dinv[i] = di;
    x[i] = 0.0;
    r[i] = bi;
    p[i] = di * bi;
    rz = fma(bi, di * bi, rz);
    bb = fma(bi, bi, bb);
  }
  rz = block_sum(rz);
  bb = block_sum(bb);
  if (threadIdx.x == 0) {
    part[RB + blockIdx.x] = rz;
    part[2 * RB + blockIdx.x] = bb;
  }
  if (last_block(&sc->done)) {
    const double rz_t = sum_partials(part, RB);
    const double bb_t = sum_partials(part, 2 * RB);
    if (threadIdx.x == 0) {
      sc->rz = rz_t;
      sc->bb = bb_t;
      sc->rr = bb_t;
      sc->done = 0;
    }
  }
}

// The solver keeps H in a slot-major ELL copy made once per solve: slot u of
// row i at u n + i (column -1 past the row's end), W = the longest row.  A
// warp's loads of slot u are then contiguous.  Rows of the condensed system
// hold 4 or 7 entries, so the copy costs ~W/7 of the CSR bytes.
constexpr int kEllMaxWidth = 16;  // wider rows keep the CSR kernel

__global__ void k_row_width(int64_t n, const int32_t* __restrict__ rowptr, unsigned* __restrict__ wmax) {
  unsigned w = 0;
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)RB * RT)
    w = max(w, (unsigned)(rowptr[i + 1] - rowptr[i]));
  for (int o = 16; o > 0; o >>= 1) w = max(w, __shfl_down_sync(0xffffffffu, w, o));
  if ((threadIdx.x & 31) == 0) atomicMax(wmax, w);
}

__global__ void k_to_ell(int64_t n, int W, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                         const double* __restrict__ val, int32_t* __restrict__ ecol, double* __restrict__ eval) {
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)RB * RT) {
    const int j0 = rowptr[i], len = rowptr[i + 1] - j0;
    for (int u = 0; u < W; ++u) {
      ecol[u * n + i] = u < len ? colind[j0 + u] : -1;
      eval[u * n + i] = u < len ? val[j0 + u] : 0.0;
    }
  }
}

// q = H p and p.q (ELL copy, one thread per row; the row sum is the fma chain
// in column order); the last block sets alpha = r.z / p.q.
template <int W>
__global__ void __launch_bounds__(RT) k_spmv_dot_ell(int64_t n, int w, const int32_t* __restrict__ ecol,
                                                     const double* __restrict__ eval, const double* __restrict__ p,
                                                     double* __restrict__ q, double* __restrict__ part,
                                                     Scalars* __restrict__ sc) {
  double pq = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)RB * RT) {
    int c[W];
    double v[W];
#pragma unroll
    for (int u = 0; u < W; ++u) {
      c[u] = u < w ? __ldcs(ecol + u * n + i) : -1;
      v[u] = u < w ? __ldcs(eval + u * n + i) : 0.0;
    }
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < W; ++u)
      if (c[u] >= 0) s = fma(v[u], __ldg(p + c[u]), s);
    q[i] = s;
    pq = fma(__ldg(p + i), s, pq);
  }
  pq = block_sum(pq);
  if (threadIdx.x == 0) part[blockIdx.x] = pq;
  if (last_block(&sc->done)) {
    const double pq_t = sum_partials(part, 0);
    if (threadIdx.x == 0) {
      sc->pq = pq_t;
      sc->alpha = pq_t > 0.0 ? sc->rz / pq_t : 0.0;
      sc->done = 0;
    }
  }
}

// The same on the CSR arrays, for rows wider than kEllMaxWidth: one thread per
// row, the first 8 values and columns loaded at once (predicated) before the
// gathers, longer rows finished in a loop.
__global__ void __launch_bounds__(RT) k_spmv_dot(int64_t n, const int32_t* __restrict__ rowptr,
                                                 const int32_t* __restrict__ colind, const double* __restrict__ val,
                                                 const double* __restrict__ p, double* __restrict__ q,
                                                 double* __restrict__ part, Scalars* __restrict__ sc) {
  double pq = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)RB * RT) {
    const int j0 = __ldg(rowptr + i), j1 = __ldg(rowptr + i + 1);
    const int len = j1 - j0;
    int c[8];
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      c[u] = u < len ? __ldg(colind + j0 + u) : 0;
      v[u] = u < len ? __ldg(val + j0 + u) : 0.0;
    }
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (u < len) s = fma(v[u], __ldg(p + c[u]), s);
    for (int j = j0 + 8; j < j1; ++j) s = fma(__ldg(val + j), __ldg(p + __ldg(colind + j)), s);
    q[i] = s;
    pq = fma(__ldg(p + i), s, pq);
  }
  pq = block_sum(pq);
  if (threadIdx.x == 0) part[blockIdx.x] = pq;
  if (last_block(&sc->done)) {
    const double pq_t = sum_partials(part, 0);
    if (threadIdx.x == 0) {
      sc->pq = pq_t;
      sc->alpha = pq_t > 0.0 ? sc->rz / pq_t : 0.0;
      sc->done = 0;
    }
  }
}

// x += alpha p, r -= alpha q (pairs of entries per 16-byte access), and the
// sums r.r and (Jacobi, JAC) r.z with z = dinv r; the last block sets rr and
// (JAC) beta = r.z_new / r.z.  With another preconditioner z and beta come
// from its application.
template <bool VEC, bool JAC>
__global__ void __launch_bounds__(RT) k_update(int64_t n, double* __restrict__ x, double* __restrict__ r,
                                               const double* __restrict__ p, const double* __restrict__ q,
                                               const double* __restrict__ dinv, Scalars* __restrict__ sc,
                                               double* __restrict__ part) {
  const double alpha = sc->alpha;
  double rz = 0.0, rr = 0.0;
  const int64_t stride = (int64_t)RB * RT;
  if (VEC) {  // x 16-byte aligned; r, p, q, dinv always are
    const int64_t n2 = n / 2;
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n2; i += stride) {
      const double2 xi = reinterpret_cast<const double2*>(x)[i], pi = reinterpret_cast<const double2*>(p)[i];
      const double2 qi = reinterpret_cast<const double2*>(q)[i], ri = reinterpret_cast<const double2*>(r)[i];
      const double2 di = JAC ? reinterpret_cast<const double2*>(dinv)[i] : make_double2(0.0, 0.0);
      const double2 xo = make_double2(fma(alpha, pi.x, xi.x), fma(alpha, pi.y, xi.y));
      const double2 ro = make_double2(fma(-alpha, qi.x, ri.x), fma(-alpha, qi.y, ri.y));
      __stcs(reinterpret_cast<double2*>(x) + i, xo);
      reinterpret_cast<double2*>(r)[i] = ro;
      if (JAC) {
        rz = fma(ro.x, di.x * ro.x, rz);
        rz = fma(ro.y, di.y * ro.y, rz);
      }
      rr = fma(ro.x, ro.x, rr);
      rr = fma(ro.y, ro.y, rr);
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
      const int64_t i = n - 1;
      x[i] = fma(alpha, p[i], x[i]);
      const double ri = fma(-alpha, q[i], r[i]);
      r[i] = ri;
      if (JAC) rz = fma(ri, dinv[i] * ri, rz);
      rr = fma(ri, ri, rr);
    }
  } else {
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += stride) {
      x[i] = fma(alpha, p[i], x[i]);
      const double ri = fma(-alpha, q[i], r[i]);
      r[i] = ri;
      if (JAC) rz = fma(ri, dinv[i] * ri, rz);
      rr = fma(ri, ri, rr);
    }
  }
  rz = block_sum(rz);
  rr = block_sum(rr);
  if (threadIdx.x == 0) {
    part[RB + blockIdx.x] = rz;
    part[2 * RB + blockIdx.x] = rr;
  }
  if (last_block(&sc->done)) {
    const double rz_t = JAC ? sum_partials(part, RB) : 0.0;
    const double rr_t = sum_partials(part, 2 * RB);
    if (threadIdx.x == 0) {
      if (JAC) {
        const double rz_old = sc->rz;
        sc->beta = rz_old > 0.0 ? rz_t / rz_old : 0.0;
        sc->rz = rz_t;
      }
      sc->rr = rr_t;
      sc->done = 0;
    }
  }
}

// p = z + beta p for a preconditioned residual z held in memory.
__global__ void __launch_bounds__(RT) k_direction_z(int64_t n, double* __restrict__ p, const double* __restrict__ z,
                                                    const Scalars* __restrict__ sc) {
  const double beta = sc->beta;
  const int64_t n2 = (n + 1) / 2;  // vectors are padded to an even length
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n2; i += (int64_t)RB * RT) {
    const double2 pi = reinterpret_cast<const double2*>(p)[i], zi = reinterpret_cast<const double2*>(z)[i];
    reinterpret_cast<double2*>(p)[i] = make_double2(fma(beta, pi.x, zi.x), fma(beta, pi.y, zi.y));
  }
}

// p = dinv r + beta p (all workspace vectors: 16-byte pairs).
__global__ void __launch_bounds__(RT) k_direction(int64_t n, double* __restrict__ p, const double* __restrict__ r,
                                                  const double* __restrict__ dinv, const Scalars* __restrict__ sc) {
  const double beta = sc->beta;
  const int64_t n2 = (n + 1) / 2;  // vectors are padded to an even length
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n2; i += (int64_t)RB * RT) {
    const double2 pi = reinterpret_cast<const double2*>(p)[i], ri = reinterpret_cast<const double2*>(r)[i];
    const double2 di = reinterpret_cast<const double2*>(dinv)[i];
    reinterpret_cast<double2*>(p)[i] = make_double2(fma(beta, pi.x, di.x * ri.x), fma(beta, pi.y, di.y * ri.y));
  }
}

// H in the solver: the ELL copy when its rows are at most kEllMaxWidth wide.
struct Matrix {
  const int32_t *rowptr, *colind;
  const double* values;
  int w;  // ELL width, 0 = use the CSR arrays
  const int32_t* ecol;
  const double* eval;
};

inline void launch_spmv_dot(int64_t n, const Matrix& A, const double* p, double* q, double* part, Scalars* sc,
                            cudaStream_t s) {
  if (A.w == 0) k_spmv_dot<<<RB, RT, 0, s>>>(n, A.rowptr, A.colind, A.values, p, q, part, sc);
  else if (A.w <= 4) k_spmv_dot_ell<4><<<RB, RT, 0, s>>>(n, A.w, A.ecol, A.eval, p, q, part, sc);
  else if (A.w <= 7) k_spmv_dot_ell<7><<<RB, RT, 0, s>>>(n, A.w, A.ecol, A.eval, p, q, part, sc);
  else k_spmv_dot_ell<kEllMaxWidth><<<RB, RT, 0, s>>>(n, A.w, A.ecol, A.eval, p, q, part, sc);
}

// one PCG iteration: 3 launches (Jacobi, z = dinv r fused), or 5 with the
// Schwarz preconditioner P (z kept in the dinv vector, y its scratch)
inline cudaError_t pcg_iteration(int64_t n, const Matrix& A, double* x, double* r, double* p, double* q,
                                 double* dinv, double* part, Scalars* sc, const ph_schwarz* P, double* y,
                                 cudaStream_t s) {
  launch_spmv_dot(n, A, p, q, part, sc, s);
  const bool vec = (reinterpret_cast<uintptr_t>(x) & 15) == 0;
  if (!P) {
    if (vec) k_update<true, true><<<RB, RT, 0, s>>>(n, x, r, p, q, dinv, sc, part);
    else k_update<false, true><<<RB, RT, 0, s>>>(n, x, r, p, q, dinv, sc, part);
    k_direction<<<RB, RT, 0, s>>>(n, p, r, dinv, sc);
    return ph::launched(3);
  }
  if (vec) k_update<true, false><<<RB, RT, 0, s>>>(n, x, r, p, q, dinv, sc, part);
  else k_update<false, false><<<RB, RT, 0, s>>>(n, x, r, p, q, dinv, sc, part);
  cudaError_t e = ph::launched(2);
  if (e == cudaSuccess) e = schwarz_apply(P, r, dinv, y, part, sc, false, s);
  if (e == cudaSuccess) {
    k_direction_z<<<RB, RT, 0, s>>>(n, p, dinv, sc);
    e = ph::launched();
  }
  return e;
}

// The solve proper on a given workspace (shared by both entry points).
// ell_ok: the solve may allocate its ELL copy of H (not in the allocation-free
// entry point).  P: Schwarz preconditioner (y: its scratch of P->nmem
// doubles), or null for Jacobi.
ph_status pcg_run(int64_t n, const int32_t* rowptr, const int32_t* colind, const double* values, const double* b,
                  double* x, double rtol, int32_t maxit, int32_t* iters, double* relres, double* work,
                  cudaStream_t s, bool ell_ok, const ph_schwarz* P = nullptr, double* y = nullptr) {
  const size_t nv = vec_stride(n);
  double *r = work, *p = r + nv, *q = p + nv, *dinv = q + nv, *part = dinv + nv;
  Scalars* sc = reinterpret_cast<Scalars*>(part + kPart);
  Scalars h;
  int it = 0;
  Matrix A{rowptr, colind, values, 0, nullptr, nullptr};
  void* ell = nullptr;
  cudaError_t e = cudaMemsetAsync(sc, 0, sizeof(Scalars), s);
  if (e == cudaSuccess && ell_ok) {  // width of the longest row (read at the first synchronisation below)
    k_row_width<<<RB, RT, 0, s>>>(n, rowptr, &sc->done);
    e = ph::launched();
  }
  // padding entries stay zero so the pairwise direction update is defined
  if (e == cudaSuccess && nv > (size_t)n) e = cudaMemsetAsync(p + n, 0, sizeof(double) * (nv - n), s);
  if (e == cudaSuccess && nv > (size_t)n) e = cudaMemsetAsync(r + n, 0, sizeof(double) * (nv - n), s);
  if (e == cudaSuccess && nv > (size_t)n) e = cudaMemsetAsync(dinv + n, 0, sizeof(double) * (nv - n), s);
  if (e == cudaSuccess && ell_ok) e = cudaMemcpyAsync(&h, sc, sizeof h, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && ell_ok) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && ell_ok && h.done <= (unsigned)kEllMaxWidth && h.done > 0) {
    const int w = (int)h.done;
    e = ph::alloc_bytes(&ell, (sizeof(double) + sizeof(int32_t)) * (size_t)w * (size_t)n + 16, s);
    if (e == cudaSuccess) {
      double* ev = static_cast<double*>(ell);
      int32_t* ec = reinterpret_cast<int32_t*>(ev + (size_t)w * n);
      k_to_ell<<<RB, RT, 0, s>>>(n, w, rowptr, colind, values, ec, ev);
      e = ph::launched();
      A = Matrix{rowptr, colind, values, w, ec, ev};
    }
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(&sc->done, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) {
    k_pcg_init<<<RB, RT, 0, s>>>(n, rowptr, colind, values, b, x, r, p, dinv, part, sc);
    e = ph::launched();
  }
  if (e == cudaSuccess && P) {  // z = M b, p = z
    e = schwarz_apply(P, r, dinv, y, part, sc, true, s);
    if (e == cudaSuccess) {
      k_direction_z<<<RB, RT, 0, s>>>(n, p, dinv, sc);
      e = ph::launched();
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, sc, sizeof h, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess || h.bad) {
    if (ell) ph::free_async(ell, s);
    return e != cudaSuccess ? ph::cuda_status(e, "pcg") : PH_ERR_ARG;
  }
  const double bnorm = sqrt(h.bb);
  double res = bnorm;
  while (res > rtol * bnorm && it < maxit) {
    const int batch = (maxit - it) < 8 ? (maxit - it) : 8;
    for (int i = 0; i < batch && e == cudaSuccess; ++i)
      e = pcg_iteration(n, A, x, r, p, q, dinv, part, sc, P, y, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, sc, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      if (ell) ph::free_async(ell, s);
      return ph::cuda_status(e, "pcg");
    }
    it += batch;
    res = sqrt(h.rr);
    if (iters) *iters = it;
    if (h.pq <= 0.0 && res > rtol * bnorm) break;  // breakdown (H not SPD)
  }
  if (ell) ph::free_async(ell, s);
  if (iters) *iters = it;
  if (relres) *relres = bnorm > 0.0 ? res / bnorm : 0.0;
  return res > rtol * bnorm ? PH_ERR_NOT_CONVERGED : PH_OK;
}

}  // namespace

using namespace ph;

extern "C" ph_status ph_solve_pcg(int64_t n, const int32_t* rowptr, const int32_t* colind, const double* values,
                                  const double* b, double* x, double rtol, int32_t maxit, int32_t* iters,
                                  double* relres, void* stream) {
  if (iters) *iters = 0;
  if (relres) *relres = 0.0;
  if (n < 0 || !(rtol >= 0.0) || maxit < 0) return PH_ERR_ARG;
  if (n == 0) return PH_OK;
  if (!rowptr || !colind || !values || !b || !x) return PH_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  double* work = nullptr;
  cudaError_t e = alloc(&work, workspace_doubles(n), s);
  if (e != cudaSuccess) return cuda_status(e, "pcg alloc");
  const ph_status st = pcg_run(n, rowptr, colind, values, b, x, rtol, maxit, iters, relres, work, s, true);
  free_async(work, s);
  return st;
}

extern "C" ph_status ph_solve_pcg_schwarz(const ph_mesh* m, const double* values, const ph_schwarz* P,
                                          const double* b, double* x, double rtol, int32_t maxit, int32_t* iters,
                                          double* relres, void* stream) {
  if (iters) *iters = 0;
  if (relres) *relres = 0.0;
  if (!m || !P || P->L != m->L || !(rtol >= 0.0) || maxit < 0) return PH_ERR_ARG;
  const int64_t n = m->L;
  if (n == 0) return PH_OK;
  if (!values || !b || !x) return PH_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  double* work = nullptr;
  const size_t wd = workspace_doubles(n);
  cudaError_t e = alloc(&work, wd + (size_t)P->nmem, s);
  if (e != cudaSuccess) return cuda_status(e, "pcg alloc");
  const ph_status st =
      pcg_run(n, m->rowptr, m->colind, values, b, x, rtol, maxit, iters, relres, work, s, true, P, work + wd);
  free_async(work, s);
  return st;
}

// ---------------------------------------------------------------------------
// Iterative refinement: the solve of H x = b to fp64 accuracy.  A plain fp64
// solve stops at an error of about cond(H) eps (~3e-9 on the jittered
// checkerboard workload); refining with a residual computed in double-word
// arithmetic takes x to the fp64 rounding of the exact solution of the system
// as given (Wilkinson's iterative refinement with an extra-precise residual).
// ---------------------------------------------------------------------------
namespace {

// Knuth's TwoSum (s + e = a + b exactly) and the fma split of a product
// (p + e = a b exactly).
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// r = b - H x: each row's sum is accumulated as an unevaluated pair (sum,
// compensation), the products split exactly by fma (Ogita, Rump and Oishi's
// Dot2), so r is as accurate as a sum formed in twice the precision and
// rounded once.
__global__ void __launch_bounds__(RT) k_residual_dw(int64_t n, const int32_t* __restrict__ rowptr,
                                                    const int32_t* __restrict__ colind,
                                                    const double* __restrict__ val, const double* __restrict__ x,
                                                    const double* __restrict__ b, double* __restrict__ r) {
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)RB * RT) {
    double sh = b[i], sl = 0.0;
    for (int j = rowptr[i]; j < rowptr[i + 1]; ++j) {
      const double v = val[j], xv = x[colind[j]];
      const double p = v * xv, pe = fma(v, xv, -p);
      double t, te;
      two_sum(sh, -p, t, te);
      sh = t;
      sl += te - pe;
    }
    r[i] = sh + sl;
  }
}

// x += d, with the sums d.d and x.x (new x) in a fixed order; the last block
// stores them in sc->pq (d.d) and sc->rr (x.x).
__global__ void __launch_bounds__(RT) k_add_correction(int64_t n, double* __restrict__ x,
                                                       const double* __restrict__ d, double* __restrict__ part,
                                                       Scalars* __restrict__ sc) {
  double dd = 0.0, xx = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)RB * RT) {
    const double di = d[i], xi = x[i] + di;
    x[i] = xi;
    dd = fma(di, di, dd);
    xx = fma(xi, xi, xx);
  }
  dd = block_sum(dd);
  xx = block_sum(xx);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = dd;
    part[RB + blockIdx.x] = xx;
  }
  if (last_block(&sc->done)) {
    const double dd_t = sum_partials(part, 0);
    const double xx_t = sum_partials(part, RB);
    if (threadIdx.x == 0) {
      sc->pq = dd_t;
      sc->rr = xx_t;
      sc->done = 0;
    }
  }
}

}  // namespace

extern "C" ph_status ph_solve_refined(const ph_mesh* m, const double* values, const ph_schwarz* P, const double* b,
                                      double* x, double tol, double inner_rtol, int32_t max_steps, int32_t maxit,
                                      int32_t* steps, int32_t* iters, double* correction, void* stream) {
  if (steps) *steps = 0;
  if (iters) *iters = 0;
  if (correction) *correction = 0.0;
  if (!m || (P && P->L != m->L) || !(tol >= 0.0) || !(inner_rtol >= 0.0) || max_steps < 1 || maxit < 0)
    return PH_ERR_ARG;
  const int64_t n = m->L;
  if (n == 0) return PH_OK;
  if (!values || !b || !x) return PH_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t wd = workspace_doubles(n), nv = vec_stride(n);
  // PCG workspace, its Schwarz scratch, then r, d, partial sums and scalars
  const size_t total = wd + (P ? (size_t)P->nmem : 0) + 2 * nv + kPart + (sizeof(Scalars) + 7) / 8;
  double* work = nullptr;
  cudaError_t e = alloc(&work, total, s);
  if (e != cudaSuccess) return cuda_status(e, "refine alloc");
  double* y = work + wd;
  double* r = y + (P ? P->nmem : 0);
  double* d = r + nv;
  double* part = d + nv;
  Scalars* sc = reinterpret_cast<Scalars*>(part + kPart);
  ph_status st = PH_OK;
  int total_it = 0, step = 0;
  double corr = INFINITY;
  e = cudaMemsetAsync(x, 0, sizeof(double) * n, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(sc, 0, sizeof(Scalars), s);
  while (e == cudaSuccess && step < max_steps) {
    ++step;
    int32_t it = 0;
    // correction equation H d = r; an inner solve that stops at its
    // iteration cap still improves x, so only other errors end the loop
    const ph_status inner = P ? pcg_run(n, m->rowptr, m->colind, values, r, d, inner_rtol, maxit, &it, nullptr,
                                        work, s, true, P, y)
                              : pcg_run(n, m->rowptr, m->colind, values, r, d, inner_rtol, maxit, &it, nullptr,
                                        work, s, true);
    total_it += it;
    if (inner != PH_OK && inner != PH_ERR_NOT_CONVERGED) {
      st = inner;
      break;
    }
    k_add_correction<<<RB, RT, 0, s>>>(n, x, d, part, sc);
    e = launched();
    Scalars h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, sc, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) break;
    corr = h.rr > 0.0 ? sqrt(h.pq / h.rr) : 0.0;
    if (corr <= tol) break;
    k_residual_dw<<<RB, RT, 0, s>>>(n, m->rowptr, m->colind, values, x, b, r);
    e = launched();
  }
  free_async(work, s);
  if (steps) *steps = step;
  if (iters) *iters = total_it;
  if (correction) *correction = corr;
  if (e != cudaSuccess) return cuda_status(e, "ph_solve_refined");
  if (st != PH_OK) return st;
  return corr <= tol ? PH_OK : PH_ERR_NOT_CONVERGED;
}

// y = H x
__global__ void k_spmv(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                       const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int j = rowptr[i]; j < rowptr[i + 1]; ++j) s = fma(val[j], x[colind[j]], s);
  y[i] = s;
}

extern "C" ph_status ph_spmv(int64_t n, const int32_t* rowptr, const int32_t* colind, const double* values,
                             const double* x, double* y, void* stream) {
  if (n < 0) return PH_ERR_ARG;
  if (n == 0) return PH_OK;
  if (!rowptr || !colind || !values || !x || !y) return PH_ERR_ARG;
  k_spmv<<<grid_for(n), kThreads, 0, (cudaStream_t)stream>>>(n, rowptr, colind, values, x, y);
  return cuda_status(launched(), "ph_spmv");
}

// ---------------------------------------------------------------------------
// ph_solve_pcg_noalloc: the iteration above with its workspace in a fixed
// device array instead of the library's pool, for callers that must not
// allocate device memory.  It reuses the kernels above unchanged.
// ---------------------------------------------------------------------------
#include <string.h>

#include <mutex>

// r, p, q, dinv (4 vectors of PH_PCG_NOALLOC_MAX_N doubles, a multiple of 32),
// partial sums and scalars: the layout of workspace_doubles().
static_assert(PH_PCG_NOALLOC_MAX_N % 32 == 0, "vector stride");
static constexpr size_t kNoAllocDoubles = 4 * (size_t)PH_PCG_NOALLOC_MAX_N + kPart + (sizeof(Scalars) + 7) / 8;
static __device__ __align__(256) double g_pcg_noalloc_work[kNoAllocDoubles];

static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[64];

// Device address of g_pcg_noalloc_work on the current device, looked up once per
// device (the host-side symbol is only a stand-in and must not reach a kernel).
static ph_status noalloc_workspace(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "ph_solve_pcg_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= 64) {
    ph::set_error_text("ph_solve_pcg_noalloc: device index >= 64 (the workspace address table holds 64 devices)");
    return PH_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_pcg_noalloc_work);
    if (e != cudaSuccess) return cuda_status(e, "ph_solve_pcg_noalloc: cudaGetSymbolAddress");
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return PH_OK;
}

extern "C" ph_status ph_solve_pcg_noalloc(int64_t n, const int32_t* rowptr, const int32_t* colind,
                                          const double* values, const double* b, double* x, double rtol,
                                          int32_t maxit, int32_t* iters, double* relres, void* stream) {
  if (iters) *iters = 0;
  if (relres) *relres = 0.0;
  if (n < 0 || !(rtol >= 0.0) || maxit < 0) return PH_ERR_ARG;
  if (n > PH_PCG_NOALLOC_MAX_N) {
    ph::set_error_text("ph_solve_pcg_noalloc: n exceeds PH_PCG_NOALLOC_MAX_N (the fixed workspace)");
    return PH_ERR_ARG;
  }
  if (n == 0) return PH_OK;
  if (!rowptr || !colind || !values || !b || !x) return PH_ERR_ARG;
  double* work = nullptr;
  ph_status st = noalloc_workspace(&work);
  if (st != PH_OK) return st;
  return pcg_run(n, rowptr, colind, values, b, x, rtol, maxit, iters, relres, work, (cudaStream_t)stream, false);
}
