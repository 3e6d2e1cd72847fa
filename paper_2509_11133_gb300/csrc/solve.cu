// Jacobi-preconditioned conjugate gradients for the condensed face system
// H Lambda = rhs (Eq. schur; the paper solves it with MATLAB's backslash).
// All reductions use a fixed grid and a fixed summation order, so repeated
// solves are bitwise reproducible.
#include <math.h>

#include "ph_internal.cuh"

namespace {

constexpr int RT = 256;   // threads per block
constexpr int RB = 1216;  // blocks (8 x 152 SMs) for vector kernels and partial sums

struct Scalars {
  double rz, pq, alpha, beta, rr, bb, rz_next;
};

// Workspace of one solve (doubles): r, p, q, dinv (4 n), then the partial sums
// part[0, RB) = p.q, part[RB, 2RB) = r.z, part[2RB, 3RB) = r.r, then Scalars
// and a flag word.
constexpr size_t kPart = 3 * (size_t)RB;

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
  return r;  // valid in thread 0
}

// Sum of part[off, off + RB) in a fixed order (every caller gets the same value).
__device__ __forceinline__ double sum_partials(const double* __restrict__ part, int off) {
  double v = 0.0;
  for (int i = threadIdx.x; i < RB; i += RT) v += part[off + i];
  return block_sum(v);
}

__global__ void __launch_bounds__(RT) k_pcg_init(int64_t n, const int32_t* __restrict__ rowptr,
                                                 const int32_t* __restrict__ colind, const double* __restrict__ val,
                                                 const double* __restrict__ b, double* __restrict__ x,
                                                 double* __restrict__ r, double* __restrict__ p,
                                                 double* __restrict__ dinv, double* __restrict__ part,
                                                 unsigned* __restrict__ bad) {
  double rz = 0.0, bb = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)RB * RT) {
    double d = 0.0;
    for (int j = rowptr[i]; j < rowptr[i + 1]; ++j)
      if (colind[j] == i) d = val[j];
    if (!(d > 0.0)) atomicOr(bad, 1u);
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
}

__global__ void __launch_bounds__(RT) k_init_scalars(const double* __restrict__ part, Scalars* sc) {
  const double rz = sum_partials(part, RB);
  const double bb = sum_partials(part, 2 * RB);
  if (threadIdx.x == 0) {
    sc->rz = rz;
    sc->rz_next = rz;
    sc->bb = bb;
    sc->rr = bb;
  }
}

// q = H p and the partial sums of p.q.  Block 0 first publishes the r.z of the
// previous iteration (read by k_update, which runs after this kernel).
__global__ void __launch_bounds__(RT) k_spmv_dot(int64_t n, const int32_t* __restrict__ rowptr,
                                                 const int32_t* __restrict__ colind, const double* __restrict__ val,
                                                 const double* __restrict__ p, double* __restrict__ q,
                                                 double* __restrict__ part, Scalars* __restrict__ sc) {
  if (blockIdx.x == 0 && threadIdx.x == 0) sc->rz = sc->rz_next;
  double pq = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)RB * RT) {
    double s = 0.0;
    for (int j = rowptr[i]; j < rowptr[i + 1]; ++j) s = fma(val[j], p[colind[j]], s);
    q[i] = s;
    pq = fma(p[i], s, pq);
  }
  pq = block_sum(pq);
  if (threadIdx.x == 0) part[blockIdx.x] = pq;
}

// alpha = r.z / p.q (every block reduces the p.q partials itself), then
// x += alpha p, r -= alpha q, and the partial sums of r.z (z = dinv r), r.r.
__global__ void __launch_bounds__(RT) k_update(int64_t n, double* __restrict__ x, double* __restrict__ r,
                                               const double* __restrict__ p, const double* __restrict__ q,
                                               const double* __restrict__ dinv, Scalars* __restrict__ sc,
                                               double* __restrict__ part) {
  __shared__ double s_alpha;
  const double pq = sum_partials(part, 0);
  if (threadIdx.x == 0) {
    const double alpha = pq > 0.0 ? sc->rz / pq : 0.0;
    s_alpha = alpha;
    if (blockIdx.x == 0) {
      sc->pq = pq;
      sc->alpha = alpha;
    }
  }
  __syncthreads();
  const double alpha = s_alpha;
  double rz = 0.0, rr = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)RB * RT) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    rz = fma(ri, dinv[i] * ri, rz);
    rr = fma(ri, ri, rr);
  }
  rz = block_sum(rz);
  rr = block_sum(rr);
  if (threadIdx.x == 0) {
    part[RB + blockIdx.x] = rz;
    part[2 * RB + blockIdx.x] = rr;
  }
}

// beta = r.z_new / r.z (every block reduces the partials itself; sc->rz is
// only read here, the new value goes to sc->rz_next), then p = dinv r + beta p.
__global__ void __launch_bounds__(RT) k_direction(int64_t n, double* __restrict__ p, const double* __restrict__ r,
                                                  const double* __restrict__ dinv, Scalars* __restrict__ sc,
                                                  const double* __restrict__ part) {
  __shared__ double s_beta;
  const double rz = sum_partials(part, RB);
  const double rr = sum_partials(part, 2 * RB);
  if (threadIdx.x == 0) {
    const double rz_old = sc->rz;
    s_beta = rz_old > 0.0 ? rz / rz_old : 0.0;
    if (blockIdx.x == 0) {
      sc->beta = s_beta;
      sc->rr = rr;
      sc->rz_next = rz;
    }
  }
  __syncthreads();
  const double beta = s_beta;
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)RB * RT)
    p[i] = fma(beta, p[i], dinv[i] * r[i]);
}

// one PCG iteration: 3 launches
inline cudaError_t pcg_iteration(int64_t n, const int32_t* rowptr, const int32_t* colind, const double* values,
                                 double* x, double* r, double* p, double* q, const double* dinv, double* part,
                                 Scalars* sc, cudaStream_t s) {
  k_spmv_dot<<<RB, RT, 0, s>>>(n, rowptr, colind, values, p, q, part, sc);
  k_update<<<RB, RT, 0, s>>>(n, x, r, p, q, dinv, sc, part);
  k_direction<<<RB, RT, 0, s>>>(n, p, r, dinv, sc, part);
  return ph::launched(3);
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
  const size_t nvec = (size_t)n;
  const size_t bytes = sizeof(double) * (4 * nvec + kPart) + sizeof(Scalars) + 16;
  cudaError_t e = alloc_bytes(reinterpret_cast<void**>(&work), bytes, s);
  if (e != cudaSuccess) return cuda_status(e, "pcg alloc");
  double *r = work, *p = r + nvec, *q = p + nvec, *dinv = q + nvec, *part = dinv + nvec;
  Scalars* sc = reinterpret_cast<Scalars*>(part + kPart);
  unsigned* bad = reinterpret_cast<unsigned*>(sc + 1);
  ph_status st = PH_OK;
  Scalars h;
  unsigned hbad = 0;
  int it = 0;
  double bnorm = 0.0, res = 0.0;
  e = cudaMemsetAsync(bad, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) {
    k_pcg_init<<<RB, RT, 0, s>>>(n, rowptr, colind, values, b, x, r, p, dinv, part, bad);
    e = launched();
  }
  if (e == cudaSuccess) {
    k_init_scalars<<<1, RT, 0, s>>>(part, sc);
    e = launched();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, sc, sizeof h, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof hbad, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { st = cuda_status(e, "pcg"); goto done; }
  if (hbad) { st = PH_ERR_ARG; goto done; }
  bnorm = sqrt(h.bb);
  res = bnorm;
  while (res > rtol * bnorm && it < maxit) {
    const int batch = (maxit - it) < 8 ? (maxit - it) : 8;
    for (int i = 0; i < batch && e == cudaSuccess; ++i)
      e = pcg_iteration(n, rowptr, colind, values, x, r, p, q, dinv, part, sc, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, sc, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { st = cuda_status(e, "pcg"); goto done; }
    it += batch;
    res = sqrt(h.rr);
    if (h.pq <= 0.0 && res > rtol * bnorm) break;  // breakdown (H not SPD)
  }
  if (iters) *iters = it;
  if (relres) *relres = bnorm > 0.0 ? res / bnorm : 0.0;
  if (res > rtol * bnorm) st = PH_ERR_NOT_CONVERGED;
done:
  free_async(work, s);
  return st;
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

// r, p, q, dinv (4 n doubles), partial sums, scalars and the flag word.
static constexpr size_t kNoAllocDoubles = 4 * (size_t)PH_PCG_NOALLOC_MAX_N + kPart + (sizeof(Scalars) + 16 + 7) / 8;
static __device__ __align__(256) double g_pcg_noalloc_work[kNoAllocDoubles];

static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[64];

// Device address of g_pcg_noalloc_work on the current device, looked up once per
// device (the host-side symbol is only a stand-in and must not reach a kernel).
static ph_status noalloc_workspace(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "ph_solve_pcg_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= 64) return PH_ERR_ARG;
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
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nvec = (size_t)n;
  double *r = work, *p = r + nvec, *q = p + nvec, *dinv = q + nvec, *part = dinv + nvec;
  Scalars* sc = reinterpret_cast<Scalars*>(part + kPart);
  unsigned* bad = reinterpret_cast<unsigned*>(sc + 1);
  Scalars h;
  unsigned hbad = 0;
  int it = 0;
  double bnorm = 0.0, res = 0.0;
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned), s);  // the only word that must start at zero
  if (e == cudaSuccess) {
    k_pcg_init<<<RB, RT, 0, s>>>(n, rowptr, colind, values, b, x, r, p, dinv, part, bad);
    e = launched();
  }
  if (e == cudaSuccess) {
    k_init_scalars<<<1, RT, 0, s>>>(part, sc);
    e = launched();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, sc, sizeof h, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof hbad, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e, "ph_solve_pcg_noalloc");
  if (hbad) return PH_ERR_ARG;
  bnorm = sqrt(h.bb);
  res = bnorm;
  while (res > rtol * bnorm && it < maxit) {
    const int batch = (maxit - it) < 8 ? (maxit - it) : 8;
    for (int i = 0; i < batch && e == cudaSuccess; ++i)
      e = pcg_iteration(n, rowptr, colind, values, x, r, p, q, dinv, part, sc, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, sc, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e, "ph_solve_pcg_noalloc");
    it += batch;
    res = sqrt(h.rr);
    if (h.pq <= 0.0 && res > rtol * bnorm) break;
  }
  if (iters) *iters = it;
  if (relres) *relres = bnorm > 0.0 ? res / bnorm : 0.0;
  return res > rtol * bnorm ? PH_ERR_NOT_CONVERGED : PH_OK;
}
