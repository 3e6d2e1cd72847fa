/*
 * ph.h -- C ABI of the GB300 library for the lowest-order primal hybrid finite
 * element method of arXiv 2509.11133 ("Vectorized 3D mesh refinement and
 * implementation of primal hybrid FEM in MATLAB"), generalised to
 *
 *     -div(a grad u) + c u = f  in Omega,   u = u_D on Gamma_D,   a grad u . nu = g on Gamma_N,
 *
 * with a per-element coefficient a_T > 0 and a constant c > 0 (the paper has
 * a = c = 1, Section 4 Eq. eq1).  The library runs the data-parallel path of
 * the method on one GPU:
 *
 *   ph_mesh_create   face-to-tetrahedron connectivity (Section 3.3), face and
 *                    multiplier numbering, the CSR pattern of the condensed
 *                    face system and per-element geometry;
 *   ph_assemble      per-element local matrices (Section 4.2), element-wise
 *                    Schur condensation onto the face multipliers (Eq. schur,
 *                    Algorithm 1 first loop) and scatter into CSR;
 *   ph_solve_pcg     a Jacobi-preconditioned conjugate-gradient solve of the
 *                    condensed system (the paper solves it with a direct
 *                    solver; Listing SchurComplement_vectorization);
 *   ph_recover       element recovery U(T) = A(T)^-1 (B(T) + C(T)' Lambda_T)
 *                    (Algorithm 1 second loop).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Array arguments are DEVICE pointers of the current CUDA device, owned by the
 *   caller.  The library keeps no reference to them after the call returns,
 *   except that ph_mesh_create copies coord and tet into the mesh.
 * - Ids are 0-based int32.  tet is row-major nE x 4, coord row-major nC x 3.
 * - Local faces of T = [a b c d] are k = 0..3: [a b c], [a c d], [a d b],
 *   [d c b] (Section 2.2).  Face k lies opposite local vertex (3, 1, 2, 0)[k].
 * - Faces are numbered by first occurrence in (tet, local face) order
 *   (Section 3.3, FacesUp).  The tet of the first occurrence is T+ of the face
 *   (sigma = +1), the other one T- (sigma = -1); a boundary face has only T+.
 * - Multipliers are the non-Neumann faces in face order (the RFaces
 *   restriction); l(F) is the multiplier id of face F, L their number.
 * - Sign convention: the exported system H Lambda = rhs has
 *   H = C A^-1 C' (symmetric positive definite) and rhs = b_D - C A^-1 B,
 *   i.e. the negatives of the paper's S and right-hand side of Eq. schur;
 *   Lambda is the paper's.
 * - stream is a cudaStream_t (NULL = legacy default stream).  Calls that do not
 *   say otherwise only enqueue work on it and return.
 * - Every entry point returns a ph_status.  Argument errors found on the host
 *   are returned at once and nothing is enqueued.  Errors found by kernels on
 *   device data (for example a non-positive coefficient a_T) set a status word
 *   in the mesh, which ph_mesh_check returns.
 */
#ifndef PH_H
#define PH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ph_mesh ph_mesh;

typedef enum {
  PH_OK = 0,
  PH_ERR_ARG = 1,            /* invalid argument or invalid mesh data        */
  PH_ERR_DEGENERATE = 2,     /* a tetrahedron with zero (or non-finite) volume */
  PH_ERR_NONMANIFOLD = 3,    /* a face shared by more than two tetrahedra     */
  PH_ERR_OVERFLOW = 4,       /* a count exceeds the int32 index range         */
  PH_ERR_NOMEM = 5,          /* device allocation failed                      */
  PH_ERR_CUDA = 6,           /* a CUDA runtime call failed                    */
  PH_ERR_NOT_CONVERGED = 7,  /* the iterative solve hit its iteration cap     */
  PH_ERR_TIMEOUT = 8         /* a bounded device-side wait ran out            */
} ph_status;

/* Counts of a mesh.  nnz is the number of stored entries of H. */
typedef struct {
  int64_t nE, nC, nF;
  int64_t nF_interior, nF_dirichlet, nF_neumann;
  int64_t L, nnz;
} ph_info;

/*
 * Build a mesh: connectivity, numbering, CSR pattern and element geometry.
 *   coord   [nC*3] float64, vertex coordinates.
 *   tet     [nE*4] int32, vertex ids of each tetrahedron (any orientation);
 *           16-byte aligned (read as int4).
 *   neumann [nN*3] int32 vertex triples of the Neumann boundary faces (the
 *           paper's Nb, Listing 1), or NULL with nN = 0.  Every other boundary
 *           face is Dirichlet.
 * Connectivity follows Section 3.3 (FacesUp) and the jump convention of
 * Section 2.2; it is computed on the device by bucketing face keys by their
 * largest vertex (and two bits of the middle one) and matching within
 * buckets, and is bit-identical to the definition (first occurrence
 * numbering).
 * Runs in order on `stream`.  Face and CSR arrays are sized by the bounds
 * nF <= 4 nE + nN and nnz <= 16 nE + nN, so the build is enqueued at once and
 * the call blocks the host once, at the end, to read the counts and the
 * first error.
 * Errors: PH_ERR_ARG for ids out of [0, nC), repeated vertices in a tet, a
 * Neumann triple that is not a boundary face of the mesh or is listed twice,
 * a misaligned tet pointer; PH_ERR_NONMANIFOLD; PH_ERR_DEGENERATE for
 * det = 0; PH_ERR_OVERFLOW when 16 nE + nN or nC reaches 2^31 - 1; a
 * look-back wait of a scan that timed out gives PH_ERR_TIMEOUT.  On error
 * *out is NULL.
 * Release with ph_mesh_destroy.
 */
ph_status ph_mesh_create(const double* coord, int64_t nC, const int32_t* tet, int64_t nE,
                         const int32_t* neumann, int64_t nN, void* stream, ph_mesh** out);

/*
 * Build n meshes at once (not in the paper: the batched path).  The same
 * result as n ph_mesh_create calls -- each out[p] is bit-identical in every
 * array to ph_mesh_create on problem p -- from one enqueued build of the
 * problems' disjoint union and one host synchronisation, instead of n.
 *   coord[p], tet[p], neumann[p] (neumann NULL, or neumann[p] NULL with
 *   nN[p] = 0; nN itself may be NULL): DEVICE pointers of problem p, as in
 *   ph_mesh_create; nC[p], nE[p], nN[p]: host arrays of its sizes.
 *   out[p] (host array of n handles) out: the meshes, usable with every entry
 *   point.  They share one device allocation, released when the last of them
 *   is passed to ph_mesh_destroy (in any order), and one status word:
 *   ph_mesh_check on any of them reports (and clears) an error recorded by a
 *   kernel on any of them.
 * Synchronises `stream` once at the end of the union's build.  Errors as
 * ph_mesh_create for any problem (then no mesh is returned); PH_ERR_OVERFLOW
 * when the union exceeds ph_mesh_create's limits (16 sum nE + sum nN or sum nC
 * reaching 2^31 - 1).
 */
ph_status ph_mesh_create_batch(int32_t n, const double* const* coord, const int64_t* nC, const int32_t* const* tet,
                               const int64_t* nE, const int32_t* const* neumann, const int64_t* nN, void* stream,
                               ph_mesh** out);

/*
 * ph_mesh_create for the double-word path (a precision variant; the paper has
 * no counterpart): the same connectivity, numbering and CSR pattern, bit for
 * bit, but the per-element geometry record holds G_e and G_e T0^-1 as scaled
 * pairs of floats, computed in double-word arithmetic on the FP32 pipe from
 * the fp64 edge vectors (|det E|, 1/|det E| and the face areas |F| stay the
 * fp64 values: the leading terms of H and of the recovery need their last
 * bits).  Such a mesh works with ph_assemble_dw, ph_recover_factored(_dw), ph_misfit,
 * ph_adjoint_rhs and every connectivity, CSR and solver entry point; the
 * entry points that read the fp64 record (ph_assemble, ph_recover,
 * ph_adjoint_grad, ph_batch_create) return PH_ERR_ARG for it.
 */
ph_status ph_mesh_create_dw(const double* coord, int64_t nC, const int32_t* tet, int64_t nE,
                            const int32_t* neumann, int64_t nN, void* stream, ph_mesh** out);

/* Free a mesh.  Its device memory is released in `stream` order. */
ph_status ph_mesh_destroy(ph_mesh* mesh, void* stream);

/* Counts of a mesh (host-side, no synchronisation). */
ph_status ph_mesh_info(const ph_mesh* mesh, ph_info* out);

/*
 * Copy connectivity out of the mesh.  Each output may be NULL.
 *   tet_face      [nE*4] int32: face id of local face k; bit 31 set when the
 *                 tet is T- of that face (sigma = -1).
 *   face_tet      [nF*2] int32: T+, T- (-1 for a boundary face).
 *   face_vtx      [nF*3] int32: the local vertex tuple of the face in T+.
 *   face_kind     [nF]   int8:  0 interior, 1 Dirichlet, 2 Neumann.
 *   face_mult     [nF]   int32: multiplier id l(F), -1 for Neumann faces.
 *   face_centroid [nF*3] float64: (P_x + P_y + P_z)/3 in face_vtx order
 *                 (the quadrature point of the load rule, Listing StiffMassPH).
 *   face_area     [nF]   float64: |F|.
 */
ph_status ph_mesh_faces(const ph_mesh* mesh, int32_t* tet_face, int32_t* face_tet, int32_t* face_vtx,
                        int8_t* face_kind, int32_t* face_mult, double* face_centroid, double* face_area,
                        void* stream);

/*
 * Copy the CSR pattern of H: rowptr [L+1], colind [nnz] (int32).  Row l(F)
 * holds F and the non-Neumann faces of F's one or two tets, columns ascending
 * (the sparsity of sum_T P_T' S(T) P_T, Listing SchurComplement_vectorization).
 */
ph_status ph_csr_pattern(const ph_mesh* mesh, int32_t* rowptr, int32_t* colind, void* stream);

/*
 * Assemble and condense (Section 4.2-4.3, Eq. schur, Algorithm 1 first loop).
 *   a       [nE] float64 coefficient per element (> 0, finite).
 *   c       reaction constant (> 0, finite; the element solve needs c > 0).
 *   f_face  [nF] float64: f at each face centroid (face_centroid order).  The
 *           load uses the paper's 4-point face-centroid rule
 *           B_j = |T|/4 sum_k f(Ct_k) phi_j(Ct_k).
 *   uD_face [nF] float64 or NULL (= 0): u_D at Dirichlet face centroids;
 *           b_D(F) = |F| u_D(Ct_F) (Section 4.3).
 *   gN_face [nF] float64 or NULL (= 0): g at Neumann face centroids;
 *           LN_j = sum_k |F_k| g(Ct_k) phi_j(Ct_k).
 *   values  [nnz] float64 out: H in the CSR pattern of ph_csr_pattern.
 *   rhs     [L]   float64 out.
 *   factor  [nE*10] float64 out, or NULL: the element factor, i.e. the 10
 *           entries (k <= m, packed 00 01 02 03 11 12 13 22 23 33) of each
 *           element's 4x4 face-indexed block of A^-1 on the complement of the
 *           constants, divided by 9.  ph_recover_factored reuses it instead of
 *           recomputing the condensation; it is valid for this mesh and this
 *           a, c only.
 * Every entry of values and rhs is overwritten.  Each stored entry of H and
 * rhs receives at most two element contributions, so the result is bitwise
 * deterministic.  Enqueues 2 kernels; no synchronisation, no allocation.
 * Errors: PH_ERR_ARG (host) for NULL mesh/a/f_face/values/rhs or invalid c;
 * an element with invalid a_T is skipped and flags PH_ERR_ARG in the mesh
 * status (ph_mesh_check).
 */
ph_status ph_assemble(const ph_mesh* mesh, const double* a, double c, const double* f_face,
                      const double* uD_face, const double* gN_face, double* values, double* rhs,
                      double* factor, void* stream);

/*
 * ph_assemble with the element condensation kernel (the 3x3 algebra behind
 * A(T)^-1 on the complement of the constants, Eq. schur) evaluated in
 * double-word arithmetic on the FP32 pipe: pairs of floats carrying ~48
 * significant bits (Dekker's exact transforms; the error bounds of Joldes,
 * Muller and Popescu 2017), with the leading term d d'/(c|T|), |det|, |F|
 * and every sum of H and rhs kept in fp64.  A precision variant, not in the
 * paper: same arguments, outputs and error behaviour as ph_assemble, results
 * within ~1e-14 relative of it (both within 1e-12 of the exact values).  An
 * element whose reaction term dominates (c h^2 comparable to a) or whose
 * data leave the exponent range of the float pairs is condensed in fp64.
 */
ph_status ph_assemble_dw(const ph_mesh* mesh, const double* a, double c, const double* f_face,
                         const double* uD_face, const double* gN_face, double* values, double* rhs, double* factor,
                         void* stream);

/*
 * Element recovery (Algorithm 1 second loop): U(T) = A(T)^-1 (B(T) + C(T)'
 * Lambda_T), Lambda_T(k) = lambda[l(F_k)] and 0 on Neumann faces.
 *   lambda [L] float64, u [nE*4] float64 out (values of u_h at the 4 vertices
 *   of each element, broken P1).  Other arguments as in ph_assemble.
 * Enqueues 1 kernel; no synchronisation, no allocation.
 */
ph_status ph_recover(const ph_mesh* mesh, const double* a, double c, const double* f_face,
                     const double* gN_face, const double* lambda, double* u, void* stream);

/*
 * Element recovery from the element factor written by ph_assemble (same
 * result as ph_recover up to rounding; no condensation arithmetic is redone).
 *   factor [nE*10] from ph_assemble on this mesh with the same a and c.
 * Other arguments as in ph_recover.  Enqueues 1 kernel.
 */
ph_status ph_recover_factored(const ph_mesh* mesh, const double* factor, double c, const double* f_face,
                              const double* gN_face, const double* lambda, double* u, void* stream);

/*
 * ph_recover_factored with the product (Qf/9) z' of Algorithm 1's second
 * loop in double-word arithmetic (float pairs, ~48 bits) on the FP32 pipe:
 * 18 FP64 operations per element instead of 34.  z' = |T|/4 f + d Lambda,
 * its sum and U = z'sum/(c|T|) - 3 (Qf/9) z' stay fp64, so the result is
 * ph_recover_factored's to the rounding of those terms.  Works on meshes from
 * ph_mesh_create and ph_mesh_create_dw; arguments, errors and the one kernel
 * as ph_recover_factored.
 */
ph_status ph_recover_factored_dw(const ph_mesh* mesh, const double* factor, double c, const double* f_face,
                                 const double* gN_face, const double* lambda, double* u, void* stream);

/*
 * Solve H x = b for a symmetric positive definite CSR matrix (rowptr [n+1],
 * colind [nnz], values [nnz]) by conjugate gradients with the Jacobi
 * preconditioner, starting from x = 0, until ||r||_2 <= rtol ||b||_2 or
 * maxit iterations.  x [n] float64 out.  iters / relres (host pointers, may
 * be NULL) receive the iteration count and the final relative residual.
 * Allocates 5n + O(1) doubles of workspace from the library's pool and
 * synchronises `stream` every 8 iterations to test convergence.
 * Errors: PH_ERR_NOT_CONVERGED when maxit is reached (x holds the last
 * iterate); PH_ERR_ARG for a non-positive diagonal entry.
 */
ph_status ph_solve_pcg(int64_t n, const int32_t* rowptr, const int32_t* colind, const double* values,
                       const double* b, double* x, double rtol, int32_t maxit, int32_t* iters,
                       double* relres, void* stream);

/* Largest system size n accepted by ph_solve_pcg_noalloc. */
#define PH_PCG_NOALLOC_MAX_N 262144

/*
 * ph_solve_pcg_noalloc -- the same Jacobi-preconditioned CG as ph_solve_pcg
 * (same arguments, same iteration, same results), but it allocates no device
 * memory.  The paper has no counterpart to this entry point: it exists for
 * callers that cannot allocate GPU memory while they run, for example a
 * long-running service that reserves its whole memory budget at start-up or
 * runs under a fixed device-memory quota, where a mid-run cudaMalloc can fail
 * or stall.  The caller still passes the CSR matrix, b and x.
 *
 * Workspace: a fixed device array inside the library (about 8.4 MB: four
 * vectors of PH_PCG_NOALLOC_MAX_N doubles plus reduction space).  Every GPU on
 * which the library's kernels are loaded holds it until the process exits.
 * - n > PH_PCG_NOALLOC_MAX_N is rejected with PH_ERR_ARG before any GPU work;
 *   ph_last_error_message() then names the limit.
 * - The first call on a device looks up the array's device address (once per
 *   device, with that device current).  The address is kept for the life of
 *   the process: like the
 *   library's memory pools, it belongs to the device's primary context, so
 *   the library must not be used across a cudaDeviceReset.  Devices 0..63
 *   only (PH_ERR_ARG, with a message, beyond).
 * - All calls share the one array, which keeps the previous call's contents
 *   (each call re-initialises what it reads).  Calls that overlap on the GPU,
 *   from several streams or threads, race on it: serialise them.
 * Never calls cudaMalloc, cudaFree or any allocating routine.  Like
 * ph_solve_pcg, it copies the convergence test's scalars to the host and
 * waits for `stream` every 8 iterations, so it returns only when the solve is
 * done.
 */
ph_status ph_solve_pcg_noalloc(int64_t n, const int32_t* rowptr, const int32_t* colind, const double* values,
                               const double* b, double* x, double rtol, int32_t maxit, int32_t* iters,
                               double* relres, void* stream);

/*
 * Batched assembly (not in the paper): many problems, meshes of uneven size
 * each with its own coefficient field, assembled and condensed by one
 * persistent kernel (plus one kernel that clears the entries receiving atomic
 * contributions).  Each problem's values, rhs and factor are bit-identical to
 * a plain ph_assemble call on it.  A batch is not thread-safe.
 *   ph_batch_create   group n meshes (the meshes must outlive the batch).
 *   ph_batch_bind     per-problem arrays: host arrays of n DEVICE pointers
 *                     (uD_face, gN_face, factor may be NULL arrays or hold
 *                     NULL entries) and a host array c[n]; uploads a
 *                     descriptor table and synchronises `stream`.
 *   ph_batch_assemble enqueue the two kernels; no allocation, no
 *                     synchronisation (capturable).
 *   ph_batch_autotune time the candidate configurations (tiles of 256..16384
 *                     elements, 64..256 threads, 2..8 blocks per SM) `reps`
 *                     times each on the bound problems, keep the fastest and
 *                     return its time per batch in *best_ms (host).
 *   ph_batch_set_config / ph_batch_get_config  the configuration in use.
 *   ph_batch_graph_launch  on first use, capture the two launches into a CUDA
 *                     graph (instantiated once; ph_batch_set_config and the
 *                     autotuner reset it, ph_batch_bind keeps it valid since
 *                     it rewrites the descriptor table in place), then launch
 *                     the graph on `stream`.
 */
typedef struct ph_batch ph_batch;
ph_status ph_batch_create(ph_mesh* const* meshes, int32_t n, void* stream, ph_batch** out);
ph_status ph_batch_destroy(ph_batch* batch, void* stream);
ph_status ph_batch_bind(ph_batch* batch, const double* const* a, const double* c, const double* const* f_face,
                        const double* const* uD_face, const double* const* gN_face, double* const* values,
                        double* const* rhs, double* const* factor, void* stream);
ph_status ph_batch_assemble(ph_batch* batch, void* stream);
ph_status ph_batch_autotune(ph_batch* batch, int32_t reps, float* best_ms, void* stream);
ph_status ph_batch_set_config(ph_batch* batch, int32_t tile, int32_t threads, int32_t blocks_per_sm, void* stream);
ph_status ph_batch_get_config(const ph_batch* batch, int32_t* tile, int32_t* threads, int32_t* blocks_per_sm);
ph_status ph_batch_graph_launch(ph_batch* batch, void* stream);
/*
 * ph_batch_bind_recovery: add element recovery from the element factor
 * (Algorithm 1, second loop, as ph_recover_factored) to the batch: host
 * arrays of n DEVICE pointers lambda[i] [L_i] and u[i] [nE_i*4]; every
 * problem must have been bound with a factor.  ph_batch_assemble and the
 * graph then run a third persistent kernel after the assembly, and each
 * problem's u is bit-identical to ph_recover_factored on its factor.
 * lambda = NULL removes the recovery.  Synchronises `stream`; the graph is
 * rebuilt on its next launch when the recovery is added or removed.
 */
ph_status ph_batch_bind_recovery(ph_batch* batch, const double* const* lambda, double* const* u, void* stream);

/*
 * Uniform refinement on the device (Section 3.4, Listing RedRefine): every
 * tet splits into 12 (4 at the vertices, 8 joining the faces of the inner
 * octahedron to the centroid), with the edge numbering of Listing NumEdges
 * and the listing's node numbering; boundary triples (the paper's Db, Nb)
 * split 1 -> 4 at edge midpoints (refineFaces).  The result is bit-identical
 * to the listing's arithmetic ((P0+P1+P2+P3)/4 and (Pa+Pb)/2).
 *   coord [nC*3], tet [nE*4] (16-byte aligned), lists [nl*3] or NULL.
 * Synchronises `stream` once (to size the output).  Errors: PH_ERR_ARG for
 * invalid tets, a misaligned tet pointer or a list triple whose edges are not
 * edges of the mesh; PH_ERR_OVERFLOW past the int32 range.
 * ph_refined_info: refined counts (nC' = nC + nE + nEd, nE' = 12 nE,
 * nl' = 4 nl) and nEd of the input mesh.  ph_refined_copy: device copies
 * (each output may be NULL).  ph_refined_destroy: free in stream order.
 */
typedef struct ph_refined ph_refined;
ph_status ph_refine(const double* coord, int64_t nC, const int32_t* tet, int64_t nE, const int32_t* lists,
                    int64_t nl, void* stream, ph_refined** out);
ph_status ph_refined_info(const ph_refined* r, int64_t* nC, int64_t* nE, int64_t* nEd_parent, int64_t* nl);
ph_status ph_refined_copy(const ph_refined* r, double* coord, int32_t* tet, int32_t* lists, void* stream);
ph_status ph_refined_destroy(ph_refined* r, void* stream);

/*
 * Additive Schwarz preconditioner over edge patches for H (an addition: the
 * paper solves with a direct method).  Patch e holds the multipliers of the
 * faces around mesh edge e (edges numbered as Listing NumEdges), and
 *     M = sum_e R_e' (R_e H R_e')^-1 R_e,
 * applied in a fixed summation order (reproducible bit for bit).  H is
 * dominated by the elementwise terms d_T d_T' / (c|T|) (Eq. schur with
 * A^-1 = J/(c|T|) + ...), whose null space -- divergence-free face fluxes --
 * is spanned by fields supported on edge patches, so M leaves a condition
 * number growing like h^-2 instead of Jacobi's a / (c h^4).
 * ph_schwarz_create: from a mesh and the values of its assembled H
 *   (ph_assemble output; CSR pattern of the mesh).  Patch blocks wider than
 *   16 use their diagonal.  Synchronises `stream` once.  PH_ERR_ARG when a
 *   patch block is not positive definite.
 * ph_solve_pcg_schwarz: conjugate gradients on H preconditioned by P;
 *   arguments and results as ph_solve_pcg (n = L of the mesh).  P must come
 *   from the same mesh and values; concurrent solves may share P.
 * ph_schwarz_destroy: frees in stream order.
 */
typedef struct ph_schwarz ph_schwarz;
ph_status ph_schwarz_create(const ph_mesh* mesh, const double* values, void* stream, ph_schwarz** out);
ph_status ph_schwarz_destroy(ph_schwarz* P, void* stream);
ph_status ph_solve_pcg_schwarz(const ph_mesh* mesh, const double* values, const ph_schwarz* P, const double* b,
                               double* x, double rtol, int32_t maxit, int32_t* iters, double* relres, void* stream);

/*
 * Solve H Lambda = rhs to fp64 accuracy by iterative refinement (an
 * addition: the paper solves with a direct method).  A plain fp64 solve of the
 * condensed system stops at an error of about cond(H) eps, which exceeds 1e-9
 * on ill-conditioned meshes (the jittered a in {1, 1e4} checkerboard).  Here:
 *     x = 0, r = rhs;  repeat:  solve H d = r by PCG to inner_rtol;  x += d;
 *     stop when ||d|| <= tol ||x||;  r = rhs - H x,
 * with the residual's row sums accumulated in double-word arithmetic (exact
 * products by fma, compensated sums), so x converges to the fp64 rounding of
 * the exact solution of the system as given.
 *   mesh, values: the condensed system (ph_assemble output, n = L).
 *   P: Schwarz preconditioner of the same mesh and values, or NULL for Jacobi.
 *   tol: relative size of the last correction (e.g. 1e-15); inner_rtol: the
 *   PCG tolerance of each correction solve (e.g. 1e-8); max_steps >= 1
 *   refinement steps; maxit: PCG iteration cap of each correction solve.
 *   steps, iters, correction (host, may be NULL): refinement steps taken, PCG
 *   iterations in total, the last relative correction.
 * Allocates its workspace from the library's pool; synchronises `stream`
 * inside each PCG solve and once per step.  PH_ERR_NOT_CONVERGED when the
 * last correction is still above tol after max_steps (x holds the last
 * iterate).
 */
ph_status ph_solve_refined(const ph_mesh* mesh, const double* values, const ph_schwarz* P, const double* b,
                           double* x, double tol, double inner_rtol, int32_t max_steps, int32_t maxit,
                           int32_t* steps, int32_t* iters, double* correction, void* stream);

/*
 * y = H x for a CSR matrix (rowptr [n+1], colind, values) and x [n], y [n]
 * (float64 device arrays).  One kernel, no synchronisation.
 */
ph_status ph_spmv(int64_t n, const int32_t* rowptr, const int32_t* colind, const double* values, const double* x,
                  double* y, void* stream);

/*
 * Adjoint of the condensed path.  The paper has no counterpart (it computes
 * no gradients).  For the misfit
 *     J = 1/2 sum_T e_T' M(T) e_T,   e_T = U_T - U_obs,T
 * (the L2 norm of a broken P1 difference; M(T) of Eq. M(T)), the gradient with
 * respect to theta_T = log a_T follows from the adjoint of the symmetric saddle
 * system of Eq. VectorForm:
 *   1. ph_adjoint_rhs:  rhs_q = -sum_T P_T' C(T) A(T)^-1 M(T) e_T;
 *   2. solve H q = rhs_q with the H of the forward assembly (ph_solve_pcg);
 *   3. ph_adjoint_grad: grad_T = -a_T p_T' K(T) U_T with
 *      p_T = A(T)^-1 (M(T) e_T + C(T)' q_T).
 * u, u_obs [nE*4] (values at the element vertices, as ph_recover writes them);
 * factor [nE*10] from ph_assemble with the same a and c; q [L]; grad [nE].
 * ph_misfit writes J to the device scalar *J (deterministic reduction; it
 * allocates 2.4 KB of workspace from the library's pool).
 * Each call enqueues 1-2 kernels; no synchronisation.
 */
ph_status ph_misfit(const ph_mesh* mesh, const double* u, const double* u_obs, double* J, void* stream);
ph_status ph_adjoint_rhs(const ph_mesh* mesh, const double* factor, double c, const double* u, const double* u_obs,
                         double* rhs_q, void* stream);
ph_status ph_adjoint_grad(const ph_mesh* mesh, const double* a, const double* factor, double c, const double* u,
                          const double* u_obs, const double* q, double* grad, void* stream);

/*
 * Synchronise `stream` and return (then clear) the mesh's device status word:
 * PH_OK or the first error a kernel recorded since the last check.
 */
ph_status ph_mesh_check(ph_mesh* mesh, void* stream);

/* Human-readable name of a status. */
const char* ph_status_string(ph_status s);

/* Message of the last PH_ERR_CUDA / PH_ERR_NOMEM raised in this thread. */
const char* ph_last_error_message(void);

/* Number of kernels this library has launched in this process. */
int64_t ph_launch_count(void);

/*
 * One pass of the whole path from and to HOST memory: upload the mesh and
 * its data, build the mesh (Section 3.3), assemble and condense (Eq. schur,
 * Algorithm 1), recover U = A^-1(B + C' Lambda) (Algorithm 1, second loop)
 * and download the system.  Equivalent to ph_mesh_create + ph_csr_pattern +
 * ph_assemble + ph_recover_factored + copies, with the copies overlapping the
 * kernels on two library streams (data up while the mesh is built, the CSR
 * pattern down while the system is assembled, values and rhs down while U is
 * recovered).  Page-locked host buffers give full-speed, asynchronous copies;
 * pageable ones work but are staged.
 *   coord [nC*3], tet [nE*4], neumann [nN*3] or NULL: as ph_mesh_create.
 *   nF, L, nnz: the counts of the mesh these tets build (ph_host_mesh_query
 *     gives them from host arrays, with the face centroids the face data are
 *     taken at); they size the face data and the outputs, and a mismatch
 *     with the build gives PH_ERR_ARG.
 *   a [nE], c, f_face [nF], uD_face [nF] or NULL, gN_face [nF] or NULL: as
 *     ph_assemble.  lambda [L] or NULL (with u NULL): the face values for the
 *     recovery.
 *   rowptr [L+1], colind [nnz], values [nnz], rhs [L], u [nE*4] or NULL:
 *     host outputs.
 * Device memory comes from the library's pool and is released before the
 * call returns; the call returns when the outputs are on the host.  Errors as
 * the entry points it stands for.
 */
ph_status ph_assemble_host(const double* coord, int64_t nC, const int32_t* tet, int64_t nE,
                           const int32_t* neumann, int64_t nN, int64_t nF, int64_t L, int64_t nnz,
                           const double* a, double c, const double* f_face, const double* uD_face,
                           const double* gN_face, const double* lambda, int32_t* rowptr, int32_t* colind,
                           double* values, double* rhs, double* u, void* stream);

/*
 * The counts, and optionally the face centroids, of the mesh that HOST arrays
 * build: what a caller holding only host memory needs before
 * ph_assemble_host (its nF, L, nnz size the outputs, and f, u_D, g are taken
 * at the face centroids).  Uploads the mesh, builds it as ph_mesh_create
 * does (Section 3.3), and releases it.
 *   coord [nC*3], tet [nE*4], neumann [nN*3] or NULL: host arrays, as in
 *     ph_assemble_host.
 *   info (host) out: the counts (ph_mesh_info).
 *   face_centroid (host, may be NULL) out: nF rows of (P_x + P_y + P_z)/3 in
 *     face order (ph_mesh_faces); centroid_capacity rows are available, and
 *     4 nE + nN always suffice.  Fewer than nF gives PH_ERR_ARG.
 * Device memory comes from the library's pool and is released before the
 * call returns; synchronises `stream`.  Errors as ph_mesh_create.
 */
ph_status ph_host_mesh_query(const double* coord, int64_t nC, const int32_t* tet, int64_t nE, const int32_t* neumann,
                             int64_t nN, ph_info* info, double* face_centroid, int64_t centroid_capacity,
                             void* stream);

/*
 * Kernel timing, off by default.  `on` is a mask: bit 0 times k_assemble,
 * zero_values (the clearing of values and rhs), k_recover and
 * k_recover_factored; bit 1 the mesh-build kernels
 * (k_face_count, k_face_fill, k_face_match, k_face_emit, k_row_fill) and
 * the scans (k_scan); 0 switches timing off.  A timed launch
 * is bracketed by a pair of CUDA events on the stream it runs on (not while
 * that stream is being captured into a graph); the events come from a pool
 * stocked when timing is switched on.  Timing the mesh build adds host work
 * between its launches and lengthens it slightly.  ph_kernel_time waits for the recorded events
 * of the named kernel, adds their elapsed times to its running total and
 * returns the total device time in ms and the number of launches timed;
 * reset != 0 clears the total afterwards.  An unknown name returns 0, 0.
 */
ph_status ph_timing_enable(int on);
ph_status ph_kernel_time(const char* kernel, int reset, double* ms, int64_t* launches);

/*
 * Test hooks (not in the paper): they let tests exercise the error paths of
 * the library without faulting or hanging a GPU.
 *   ph_test_fail_alloc(after): the (after+1)-th device allocation from the
 *     library's pool from now on fails as if the device were out of memory
 *     (the call that made it returns PH_ERR_NOMEM and frees what it had
 *     taken); after < 0 switches the hook off.  Later allocations succeed.
 *   ph_test_scan_withhold(on): while on, the device-wide scans of
 *     ph_mesh_create (and of the Schwarz set-up) run with their tile 1 never
 *     publishing its partial sum and a look-back poll limit of 2^12, so the
 *     wait of the tiles after it runs out: they record PH_ERR_TIMEOUT in the
 *     status word and return (every wait in the scan is bounded; nothing
 *     hangs).  Scans of fewer than three tiles (4096 values each) are not
 *     affected.  Off by default; for tests only.
 *   ph_pool_in_use(bytes): (host) bytes of the current device's library pool
 *     held by live allocations (freed memory counts once its stream-ordered
 *     free has run), to check that failed calls leak nothing.
 * The hooks are process-wide and not synchronised with calls in flight on
 * other threads.
 */
ph_status ph_test_fail_alloc(int64_t after);
ph_status ph_test_scan_withhold(int on);
ph_status ph_pool_in_use(int64_t* bytes);

/*
 * Measure the FP64 pipe's throughput on the current device (not in the paper;
 * it gives the element kernels' roofline its denominator).  One kernel of
 * 8 blocks of 256 threads per SM, each thread running 16 independent chains
 * of `iters` DFMA operations, timed with a pair of CUDA events on `stream`.
 *   iters      > 0; about 4000 gives a launch of tens of milliseconds.
 *   ops_per_s  (host) out: DFMA operations per second over the whole GPU
 *              (one fused multiply-add counts as one operation).
 *   ms         (host, may be NULL) out: the launch's duration.
 * Allocates a small result buffer from the library's pool and synchronises
 * `stream`.
 */
ph_status ph_fp64_peak(int64_t iters, double* ops_per_s, double* ms, void* stream);

/*
 * y[i] = 1/x[i] with the device reciprocal the element kernels use for
 * 1/|det E| and 1/det M (a Newton iteration; within one ulp of the rounded
 * quotient, and the IEEE quotient for x outside [2^-1020, 2^1021)).  Device
 * arrays of n doubles; exposed so that its accuracy can be tested.
 */
ph_status ph_rcp(const double* x, int64_t n, double* y, void* stream);

/*
 * y[i] = sqrt(x[i])/2 with the device square root the mesh build uses for
 * the face areas |F| = |(P_z - P_x) x (P_y - P_x)|/2 (Section 4.2, C(T)):
 * a coupled Newton iteration from a single-precision seed, within one ulp of
 * the rounded sqrt(x)/2, and 0.5 * sqrt(x) for x outside [2^-960, 2^960).
 * Device arrays of n doubles; exposed so that its accuracy can be tested.
 */
ph_status ph_half_sqrt(const double* x, int64_t n, double* y, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PH_H */
