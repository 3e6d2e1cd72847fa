// One pass of the whole path from and to host memory (ph_assemble_host):
// upload, build the mesh (Section 3.3), assemble and condense (Eq. schur,
// Algorithm 1 first loop), recover the element values (Algorithm 1 second
// loop), download.  The copies run on two library streams (a pair per call
// in flight) beside the kernels on the caller's stream:
//   up:   a, f, u_D, g_N, Lambda            while the mesh is built
//   down: rowptr, colind                    while the system is assembled
//         values, rhs                       while the elements are recovered
//         U                                 last
// so a call costs about the upload of the mesh, its build, and the download
// of the system (the host link, ~0.2 TB/s each way, binds).  Calls from
// several host threads, each on its own stream, overlap one call's download
// with the next one's build.
#include <mutex>
#include <utility>
#include <vector>

#include "ph_internal.cuh"

using namespace ph;

namespace {

// Copy-stream pairs per device, one pair per call in flight, so that
// concurrent calls (several host threads) do not queue behind each other.
std::mutex g_mu;
std::vector<std::pair<cudaStream_t, cudaStream_t>> g_free[64];

cudaError_t acquire_streams(int dev, cudaStream_t* up, cudaStream_t* down) {
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_free[dev].empty()) {
      *up = g_free[dev].back().first;
      *down = g_free[dev].back().second;
      g_free[dev].pop_back();
      return cudaSuccess;
    }
  }
  cudaError_t e = cudaStreamCreateWithFlags(up, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(down, cudaStreamNonBlocking);
  return e;
}

void release_streams(int dev, cudaStream_t up, cudaStream_t down) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_free[dev].emplace_back(up, down);
}

template <class T>
cudaError_t upload(T* d, const T* h, int64_t n, cudaStream_t s) {
  return (h && n > 0) ? cudaMemcpyAsync(d, h, sizeof(T) * n, cudaMemcpyHostToDevice, s) : cudaSuccess;
}

template <class T>
cudaError_t download(T* h, const T* d, int64_t n, cudaStream_t s) {
  return (h && n > 0) ? cudaMemcpyAsync(h, d, sizeof(T) * n, cudaMemcpyDeviceToHost, s) : cudaSuccess;
}

}  // namespace

extern "C" ph_status ph_assemble_host(const double* coord, int64_t nC, const int32_t* tet, int64_t nE,
                                      const int32_t* neumann, int64_t nN, int64_t nF, int64_t L, int64_t nnz,
                                      const double* a, double c, const double* f_face, const double* uD_face,
                                      const double* gN_face, const double* lambda, int32_t* rowptr,
                                      int32_t* colind, double* values, double* rhs, double* u, void* stream) {
  if (nC < 0 || nE < 0 || nN < 0 || nF < 0 || L < 0 || nnz < 0) return PH_ERR_ARG;
  if ((nC > 0 && !coord) || (nE > 0 && (!tet || !a)) || (nN > 0 && !neumann) || (nF > 0 && !f_face)) return PH_ERR_ARG;
  if ((L > 0 && (!rowptr || !rhs)) || (nnz > 0 && (!colind || !values)) || (u && !lambda)) return PH_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream, up = nullptr, down = nullptr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = acquire_streams(dev, &up, &down);
  if (e != cudaSuccess) return cuda_status(e, "ph_assemble_host");

  double *d_coord = nullptr, *d_a = nullptr, *d_f = nullptr, *d_uD = nullptr, *d_gN = nullptr, *d_lam = nullptr;
  double *d_values = nullptr, *d_rhs = nullptr, *d_factor = nullptr, *d_u = nullptr;
  int32_t *d_tet = nullptr, *d_neu = nullptr;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // start, uploaded, built, assembled, downloaded
  ph_mesh* m = nullptr;
  ph_status st = PH_OK;
  for (cudaEvent_t& x : ev)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
  // device buffers, stream-ordered on the caller's stream
  if (e == cudaSuccess) e = alloc(&d_coord, (size_t)(3 * nC), s);
  if (e == cudaSuccess) e = alloc(&d_tet, (size_t)(4 * nE), s);
  if (e == cudaSuccess && nN > 0) e = alloc(&d_neu, (size_t)(3 * nN), s);
  if (e == cudaSuccess) e = alloc(&d_a, (size_t)nE, s);
  if (e == cudaSuccess) e = alloc(&d_f, (size_t)nF, s);
  if (e == cudaSuccess && uD_face) e = alloc(&d_uD, (size_t)nF, s);
  if (e == cudaSuccess && gN_face) e = alloc(&d_gN, (size_t)nF, s);
  if (e == cudaSuccess && lambda) e = alloc(&d_lam, (size_t)L, s);
  if (e == cudaSuccess) e = alloc(&d_values, (size_t)nnz, s);
  if (e == cudaSuccess) e = alloc(&d_rhs, (size_t)L, s);
  if (e == cudaSuccess) e = alloc(&d_factor, (size_t)(10 * nE), s);
  if (e == cudaSuccess && u) e = alloc(&d_u, (size_t)(4 * nE), s);
  // the mesh inputs on the caller's stream; everything else on `up`
  if (e == cudaSuccess) e = upload(d_coord, coord, 3 * nC, s);
  if (e == cudaSuccess) e = upload(d_tet, tet, 4 * nE, s);
  if (e == cudaSuccess) e = upload(d_neu, neumann, 3 * nN, s);
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(up, ev[0], 0);
  if (e == cudaSuccess) e = upload(d_a, a, nE, up);
  if (e == cudaSuccess) e = upload(d_f, f_face, nF, up);
  if (e == cudaSuccess) e = upload(d_uD, uD_face, nF, up);
  if (e == cudaSuccess) e = upload(d_gN, gN_face, nF, up);
  if (e == cudaSuccess) e = upload(d_lam, lambda, L, up);
  if (e == cudaSuccess) e = cudaEventRecord(ev[1], up);
  if (e != cudaSuccess) { st = cuda_status(e, "ph_assemble_host"); goto done; }

  st = ph_mesh_create(d_coord, nC, d_tet, nE, d_neu, nN, s, &m);  // blocks the host once
  if (st != PH_OK) goto done;
  if (m->nF != nF || m->L != L || m->nnz != nnz) {
    set_error_text("ph_assemble_host: nF, L or nnz differ from the mesh built from these tets");
    st = PH_ERR_ARG;
    goto done;
  }
  // the CSR pattern goes down while the system is assembled
  e = cudaEventRecord(ev[2], s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(down, ev[2], 0);
  if (e == cudaSuccess) e = download(rowptr, m->rowptr, L + 1, down);
  if (e == cudaSuccess) e = download(colind, m->colind, nnz, down);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[1], 0);
  if (e != cudaSuccess) { st = cuda_status(e, "ph_assemble_host"); goto done; }
  st = ph_assemble(m, d_a, c, d_f, d_uD, d_gN, d_values, d_rhs, d_factor, s);
  if (st != PH_OK) goto done;
  // values and rhs go down while the elements are recovered
  e = cudaEventRecord(ev[3], s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(down, ev[3], 0);
  if (e == cudaSuccess) e = download(values, d_values, nnz, down);
  if (e == cudaSuccess) e = download(rhs, d_rhs, L, down);
  if (e != cudaSuccess) { st = cuda_status(e, "ph_assemble_host"); goto done; }
  if (u) {
    st = ph_recover_factored(m, d_factor, c, d_f, d_gN, d_lam, d_u, s);
    if (st != PH_OK) goto done;
    e = cudaEventRecord(ev[3], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(down, ev[3], 0);
    if (e == cudaSuccess) e = download(u, d_u, 4 * nE, down);
    if (e != cudaSuccess) { st = cuda_status(e, "ph_assemble_host"); goto done; }
  }

done:
  // join both copy streams into the caller's stream, free in stream order,
  // and return with the outputs on the host
  if (ev[4] && cudaEventRecord(ev[4], up) == cudaSuccess) cudaStreamWaitEvent(s, ev[4], 0);
  if (ev[4] && cudaEventRecord(ev[4], down) == cudaSuccess) cudaStreamWaitEvent(s, ev[4], 0);
  if (m) ph_mesh_destroy(m, s);
  for (void* p : {(void*)d_coord, (void*)d_tet, (void*)d_neu, (void*)d_a, (void*)d_f, (void*)d_uD, (void*)d_gN,
                  (void*)d_lam, (void*)d_values, (void*)d_rhs, (void*)d_factor, (void*)d_u})
    free_async(p, s);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess && st == PH_OK) st = cuda_status(e, "ph_assemble_host");
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  release_streams(dev, up, down);  // idle: the caller's stream waited for both
  return st;
}

// Counts (and face centroids) of the mesh that host arrays build: the query a
// caller with only host memory makes before ph_assemble_host, to size its
// outputs and evaluate f, u_D, g at the face centroids.
namespace {
__global__ void k_centroids(const double* __restrict__ coord, const int32_t* __restrict__ face_vtx, int64_t nF,
                            double* __restrict__ out) {
  const int64_t F = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (F >= nF) return;
  const double* x = coord + 3 * (int64_t)face_vtx[3 * F];
  const double* y = coord + 3 * (int64_t)face_vtx[3 * F + 1];
  const double* z = coord + 3 * (int64_t)face_vtx[3 * F + 2];
#pragma unroll
  for (int d = 0; d < 3; ++d) out[3 * F + d] = (x[d] + y[d] + z[d]) / 3.0;
}
}  // namespace

extern "C" ph_status ph_host_mesh_query(const double* coord, int64_t nC, const int32_t* tet, int64_t nE,
                                        const int32_t* neumann, int64_t nN, ph_info* info, double* face_centroid,
                                        int64_t centroid_capacity, void* stream) {
  if (!info || nC < 0 || nE < 0 || nN < 0 || centroid_capacity < 0) return PH_ERR_ARG;
  if ((nC > 0 && !coord) || (nE > 0 && !tet) || (nN > 0 && !neumann)) return PH_ERR_ARG;
  if (4 * nE + nN >= ((int64_t)1 << 31) - 1) return PH_ERR_OVERFLOW;
  cudaStream_t s = (cudaStream_t)stream;
  double* d_coord = nullptr;
  int32_t *d_tet = nullptr, *d_neu = nullptr;
  double* d_cen = nullptr;
  ph_mesh* m = nullptr;
  ph_status st = PH_OK;
  cudaError_t e = alloc(&d_coord, (size_t)(3 * nC), s);
  if (e == cudaSuccess) e = alloc(&d_tet, (size_t)(4 * nE), s);
  if (e == cudaSuccess && nN > 0) e = alloc(&d_neu, (size_t)(3 * nN), s);
  if (e == cudaSuccess) e = upload(d_coord, coord, 3 * nC, s);
  if (e == cudaSuccess) e = upload(d_tet, tet, 4 * nE, s);
  if (e == cudaSuccess) e = upload(d_neu, neumann, 3 * nN, s);
  if (e != cudaSuccess) {
    st = cuda_status(e, "ph_host_mesh_query");
  } else {
    st = ph_mesh_create(d_coord, nC, d_tet, nE, d_neu, nN, s, &m);  // blocks the host once
  }
  if (st == PH_OK) st = ph_mesh_info(m, info);
  if (st == PH_OK && face_centroid && m->nF > 0) {
    if (centroid_capacity < m->nF) {
      set_error_text("ph_host_mesh_query: face_centroid holds fewer than nF rows");
      st = PH_ERR_ARG;
    } else {
      e = alloc(&d_cen, (size_t)(3 * m->nF), s);
      if (e == cudaSuccess) {
        k_centroids<<<grid_for(m->nF), kThreads, 0, s>>>(m->coord, m->face_vtx, m->nF, d_cen);
        e = launched();
      }
      if (e == cudaSuccess) e = download(face_centroid, d_cen, 3 * m->nF, s);
      if (e != cudaSuccess) st = cuda_status(e, "ph_host_mesh_query");
    }
  }
  if (m) ph_mesh_destroy(m, s);
  for (void* p : {(void*)d_coord, (void*)d_tet, (void*)d_neu, (void*)d_cen}) free_async(p, s);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess && st == PH_OK) st = cuda_status(e, "ph_host_mesh_query");
  return st;
}

