// Internal declarations of the primal hybrid FEM library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "fp64.cuh"
#include "ph.h"

// tmult encoding: multiplier id in bits 0..30, bit 31 = Dirichlet boundary
// face; PH_NO_MULT marks a Neumann face (no multiplier).
#define PH_NO_MULT 0x7FFFFFFF
#define PH_BND_BIT 0x80000000u
#define PH_ID_MASK 0x7FFFFFFF
// Per-element geometry record (doubles): G_e = E E' (00 01 02 11 12 22),
// GT = G_e T0^-1 row-major (9), |det E|, 1/|det E|, padding.
#define PH_GEO_STRIDE 18

// Device memory shared by the meshes of one batched build (ph_mesh_create_batch):
// released when the last of them is destroyed.
struct ph_mesh_shared {
  std::atomic<int> refs;
  void* arena;  // the union mesh's arrays
  void* extra;  // per-problem row pointers and offset tables
};

struct ph_mesh {
  int device;
  ph_mesh_shared* shared;  // non-null for a mesh of a batched build (arena then unused)
  void* arena;         // one allocation holding every array below
  int64_t nE, nC, nF, nFi, nFd, nFn, L, nnz;
  double* coord;       // nC*3
  int4* tet;           // nE
  int4* tface;         // nE: face id, bit 31 = sigma < 0
  int4* tmult;         // nE: see PH_NO_MULT / PH_BND_BIT
  int4* tpos;          // nE: CSR position of the diagonal entry of row l(F_k)
  ushort4* trel;       // nE: 3 packed 4-bit offsets (m != k, ascending m) from tpos
  double* geo;         // nE*PH_GEO_STRIDE: G_e, G_e T0^-1, |det|, 1/|det|
  int2* face_tet;      // nF
  int32_t* face_vtx;   // nF*3
  int8_t* face_kind;   // nF
  int32_t* face_mult;  // nF
  double* face_area;   // nF
  int32_t* rowptr;     // L+1
  int32_t* colind;     // nnz
  int32_t* rowdiag;    // L
  unsigned int* status;  // device status word: bit s set for ph_status s
  bool geo_dw;           // geo holds the double-word record (ph_mesh_create_dw)
};

namespace ph {

extern std::atomic<int64_t> g_launches;

// Record one kernel launch and return the launch error, if any.
inline cudaError_t launched(int n = 1) {
  g_launches.fetch_add(n, std::memory_order_relaxed);
  return cudaGetLastError();
}

// Opt-in device timing of named kernels (ph_timing_enable): brackets one
// launch with CUDA events on its stream; a no-op while timing is off or the
// stream is being captured into a graph.
class KernelTimer {
 public:
  // category 1: element kernels (assembly, recovery); 2: mesh build and scans
  KernelTimer(const char* name, cudaStream_t s, unsigned category = 1);
  ~KernelTimer() { stop(); }
  KernelTimer(const KernelTimer&) = delete;
  KernelTimer& operator=(const KernelTimer&) = delete;
  void stop();  // after the launch (again at scope exit: no effect)
 private:
  const char* name_;
  cudaStream_t s_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
};

void set_error_message(const char* what, cudaError_t e);
void set_error_text(const char* text);
ph_status cuda_status(cudaError_t e, const char* what);

// Stream-ordered allocation from the library's memory pool of `device`.
cudaError_t alloc_bytes(void** p, size_t bytes, cudaStream_t s);
template <class T>
inline cudaError_t alloc(T** p, size_t n, cudaStream_t s) {
  return alloc_bytes(reinterpret_cast<void**>(p), n * sizeof(T) + (n == 0 ? 16 : 0), s);
}
void free_async(void* p, cudaStream_t s);

// Exclusive prefix sum of n non-negative int32 values into out (int32), one
// kernel; the int64 total is written to *d_total (device).  in and out may
// alias.  With d_len, only min(n, *d_len + len_add) values (a length known
// on the device) are scanned.  A look-back wait that times out sets
// PH_ERR_TIMEOUT in *status (if given) instead of hanging.
// `state` (optional): a zeroed workspace of scan_state_words(n) words; without
// it the scan allocates and clears its own.
// `mates` (optional, replaces `in`): the face mates of nmates tets (mate slot
// of each local face, see first_occurrence); value i is the number of faces
// whose first occurrence is in tet i (0 for i >= nmates), so the scan numbers
// the faces without a separate counting pass.
ph_status exclusive_scan(const int32_t* in, int32_t* out, int64_t n, int64_t* d_total, cudaStream_t s,
                         unsigned* status = nullptr, const int64_t* d_len = nullptr, int64_t len_add = 0,
                         unsigned long long* state = nullptr, const int4* mates = nullptr, int64_t nmates = 0);

// Local face slot s = 4t + k is the first occurrence of its face when its mate
// slot m is a boundary mark (m < 0) or a later slot.
__device__ __forceinline__ bool first_occurrence(int m, int s) { return m < 0 || m > s; }
__device__ __forceinline__ int first_occurrences(int4 m, int s0) {
  return first_occurrence(m.x, s0) + first_occurrence(m.y, s0 + 1) + first_occurrence(m.z, s0 + 2) +
         first_occurrence(m.w, s0 + 3);
}
size_t scan_state_words(int64_t n);

// Sub-arrays of one allocation, each starting on a 256-byte boundary.
struct Carve {
  size_t bytes = 0;
  template <class T>
  size_t take(size_t n) {
    const size_t at = bytes;
    bytes += (n * sizeof(T) + 255) & ~(size_t)255;
    return at;
  }
  template <class T>
  static T* at(void* base, size_t off) {
    return reinterpret_cast<T*>(static_cast<char*>(base) + off);
  }
};

// First error recorded in a status word (lowest code), PH_OK if none.
inline ph_status status_from_bits(unsigned bits) {
  for (int c = 1; c < 32; ++c)
    if (bits & (1u << c)) return (ph_status)c;
  return PH_OK;
}

constexpr int kThreads = 256;
inline unsigned grid_for(int64_t n, int threads = kThreads) {
  int64_t g = (n + threads - 1) / threads;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace ph

// Record an error code in a device status word.
__device__ __forceinline__ void ph_flag(unsigned* status, ph_status s) { atomicOr(status, 1u << (unsigned)s); }
