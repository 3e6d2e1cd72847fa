// Internals of the conjugate-gradient solver shared by the Jacobi and the
// Schwarz-preconditioned solves: launch shape, device scalars, deterministic
// block and grid reductions, and the Schwarz preconditioner's data.
#pragma once

#include "ph_internal.cuh"

namespace ph_pcg {

constexpr int RT = 256;   // threads per block
constexpr int RB = 1216;  // blocks (8 x 152 SMs) for vector kernels and partial sums

struct Scalars {
  double rz, pq, alpha, beta, rr, bb;
  unsigned done;  // blocks finished in the current reducing kernel (last-block detection)
  unsigned bad;   // a non-positive diagonal entry was seen
};

// Partial sums: part[0, RB) = p.q, part[RB, 2RB) = r.z, part[2RB, 3RB) = r.r.
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

// Sum of part[off, off + RB) in a fixed order (every caller gets the same
// value); the partials come from other blocks, so they bypass L1.
__device__ __forceinline__ double sum_partials(const double* __restrict__ part, int off) {
  double v = 0.0;
  for (int i = threadIdx.x; i < RB; i += RT) v += __ldcg(part + off + i);
  return block_sum(v);
}

// True in the block that finishes last (it then owns the final reduction).
// The caller's thread 0 wrote its partial before; the fence orders it before
// the count.
__device__ __forceinline__ bool last_block(unsigned* done) {
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  return s_last;
}

// z = M r for the edge-patch Schwarz preconditioner P (y: scratch of
// P->nmem doubles), with the sum r.z: init sets rz, otherwise the last block
// sets beta = r.z / rz_old and rz.  Two launches.
cudaError_t schwarz_apply(const ph_schwarz* P, const double* r, double* z, double* y, double* part, Scalars* sc,
                          bool init, cudaStream_t s);

}  // namespace ph_pcg

// Additive Schwarz preconditioner over edge patches: patch e holds the
// multipliers of the faces around edge e; M = sum_e R_e' (R_e H R_e')^-1 R_e.
// Patches are grouped by their number of members k (a patch wider than
// kSchwarzDense becomes k patches of one member: its diagonal), and within a
// group every array is slot-major (entry q of patch s at base + q count + s),
// so the threads of a warp -- consecutive patches of one group -- make
// contiguous accesses.
constexpr int kSchwarzDense = 16;  // widest patch inverted densely

struct SchwarzGroups {
  int64_t count[kSchwarzDense + 1];  // patches with k members
  int64_t first[kSchwarzDense + 2];  // index of the first patch of group k (patches ordered by k)
  int64_t mbase[kSchwarzDense + 1];  // group k in mem and y: k slots per patch
  int64_t bbase[kSchwarzDense + 1];  // group k in blk: k(k+1)/2 entries per patch
};

struct ph_schwarz {
  int device;
  int64_t L, nEd, nmem, npatch, nblk;
  SchwarzGroups g;
  int32_t* mem;    // multiplier ids, ascending within a patch
  double* blk;     // patch inverses: packed upper triangle, row-major
  int32_t* fslot;  // 3L: positions in mem (and y) of each multiplier in the patches of its face's three edges
};
