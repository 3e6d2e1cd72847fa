/*
 * ph_oracle.c -- plain CPU oracle for the lowest-order primal hybrid FEM path
 * (arXiv 2509.11133).  TEST INFRASTRUCTURE ONLY: it exists to check the CUDA
 * library.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load it; the product path never does.  It shares no code, header
 * or table with the CUDA library.
 *
 * Everything here is the paper's definitions written out, element by element:
 *   - faces: every distinct vertex set of a local face is one face, numbered
 *     by first occurrence in (tet, local face) order; the tet of the first
 *     occurrence is T+ (Section 3.3, FacesUp; the jump definition of Section 2.2);
 *   - local matrices K(T), M(T), C(T) (Eqs. K(T), M(T), C(T), Section 4.2),
 *     the face-centroid load rule and b_D, LN (Section 4.3);
 *   - element condensation S(T) = C A^-1 C', rhs(T) = b_D - C A^-1 B
 *     (Eq. schur, Algorithm 1), with the sign flipped so that the exported
 *     face system is symmetric positive definite;
 *   - recovery U(T) = A^-1 (B + C' Lambda) (Algorithm 1, second loop).
 *
 * Precision: every per-element quantity is computed in IEEE binary128
 * (_Float128) from the fp64 inputs and rounded to fp64 once at the end.  The
 * local matrix A = aK + cM has condition number ~ a/(c h^2); doing the
 * definition in fp64 would lose up to ~8 digits on fine meshes, so the oracle
 * evaluates it in quad to stay an accurate reference for fp64 results.
 */
#define __STDC_WANT_IEC_60559_TYPES_EXT__
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef _Float128 qf;

enum {
  OR_OK = 0,
  OR_ERR_ARG = 1,
  OR_ERR_DEGENERATE = 2,
  OR_ERR_NONMANIFOLD = 3,
  OR_ERR_OVERFLOW = 4,
  OR_ERR_NOMEM = 5
};

/* face kinds */
enum { KIND_INTERIOR = 0, KIND_DIRICHLET = 1, KIND_NEUMANN = 2 };

/* Local faces of T = [a b c d]: [a b c], [a c d], [a d b], [d c b] (Section 2.2). */
static const int LFACE[4][3] = {{0, 1, 2}, {0, 2, 3}, {0, 3, 1}, {3, 2, 1}};

/* phi_j at the centroid of local face k: 1/3 if vertex j lies on face k, else 0. */
static int on_face(int k, int j) {
  return LFACE[k][0] == j || LFACE[k][1] == j || LFACE[k][2] == j;
}

/* ------------------------------------------------------------------------ */
/* quad helpers                                                               */
/* ------------------------------------------------------------------------ */
static qf qabs(qf x) { return x < 0 ? -x : x; }

/* square root by Newton's (Heron's) iteration from the fp64 root */
static qf qsqrt(qf x) {
  if (x <= 0) return 0;
  qf y = (qf)sqrt((double)x);
  for (int i = 0; i < 3; ++i) y = (y + x / y) / 2;
  return y;
}

/* Solve A X = R for X (n x n, m right-hand sides) by Gaussian elimination
 * with partial pivoting.  A and R are overwritten.  Returns 0 if singular. */
static int qsolve(int n, qf A[4][4], int m, qf R[4][8]) {
  for (int col = 0; col < n; ++col) {
    int p = col;
    for (int r = col + 1; r < n; ++r)
      if (qabs(A[r][col]) > qabs(A[p][col])) p = r;
    if (A[p][col] == 0) return 0;
    if (p != col) {
      for (int j = 0; j < n; ++j) { qf t = A[p][j]; A[p][j] = A[col][j]; A[col][j] = t; }
      for (int j = 0; j < m; ++j) { qf t = R[p][j]; R[p][j] = R[col][j]; R[col][j] = t; }
    }
    for (int r = col + 1; r < n; ++r) {
      qf f = A[r][col] / A[col][col];
      for (int j = col; j < n; ++j) A[r][j] -= f * A[col][j];
      for (int j = 0; j < m; ++j) R[r][j] -= f * R[col][j];
    }
  }
  for (int col = n - 1; col >= 0; --col) {
    for (int j = 0; j < m; ++j) {
      qf s = R[col][j];
      for (int k = col + 1; k < n; ++k) s -= A[col][k] * R[k][j];
      R[col][j] = s / A[col][col];
    }
  }
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Per-element quantities (Section 4.2-4.3)                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
  qf vol;          /* |T| */
  qf grad[4][3];   /* grad lambda_i */
  qf K[4][4];      /* |T| grad_i . grad_j */
  qf M[4][4];      /* |T|/20 (I + J) */
  qf area[4];      /* |F_k| */
} geom_q;

/* Volume and barycentric gradients from G = [1 1 1 1; x; y; z]^-1 [0;I3]
 * (Eq. K(T)), K = |T| G G' (the listing's form, see the reading of the
 * printed prefactor), M (Eq. M(T)) and face areas 1/2 |(P_z-P_x) x (P_y-P_x)|
 * for the local face tuple [x y z] (Listing Multiplier). */
static int geom(const double P[4][3], geom_q* g) {
  qf Gm[4][4], R[4][8];
  for (int j = 0; j < 4; ++j) {
    Gm[0][j] = 1;
    for (int d = 0; d < 3; ++d) Gm[d + 1][j] = (qf)P[j][d];
  }
  /* det(Gm) by elimination on a copy */
  qf D[4][4];
  memcpy(D, Gm, sizeof D);
  qf det = 1;
  for (int col = 0; col < 4; ++col) {
    int p = col;
    for (int r = col + 1; r < 4; ++r)
      if (qabs(D[r][col]) > qabs(D[p][col])) p = r;
    if (D[p][col] == 0) return 0;
    if (p != col) {
      for (int j = 0; j < 4; ++j) { qf t = D[p][j]; D[p][j] = D[col][j]; D[col][j] = t; }
      det = -det;
    }
    det *= D[col][col];
    for (int r = col + 1; r < 4; ++r) {
      qf f = D[r][col] / D[col][col];
      for (int j = col; j < 4; ++j) D[r][j] -= f * D[col][j];
    }
  }
  g->vol = qabs(det) / 6;
  /* G = Gm^-1 [0 0 0; 1 0 0; 0 1 0; 0 0 1]: solve Gm X = E */
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 3; ++j) R[i][j] = (i == j + 1) ? 1 : 0;
  if (!qsolve(4, Gm, 3, R)) return 0;
  for (int i = 0; i < 4; ++i)
    for (int d = 0; d < 3; ++d) g->grad[i][d] = R[i][d];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      qf s = 0;
      for (int d = 0; d < 3; ++d) s += g->grad[i][d] * g->grad[j][d];
      g->K[i][j] = g->vol * s;
      g->M[i][j] = g->vol / 20 * ((i == j) ? 2 : 1);
    }
  for (int k = 0; k < 4; ++k) {
    const double* x = P[LFACE[k][0]];
    const double* y = P[LFACE[k][1]];
    const double* z = P[LFACE[k][2]];
    qf u[3], v[3];
    for (int d = 0; d < 3; ++d) { u[d] = (qf)z[d] - (qf)x[d]; v[d] = (qf)y[d] - (qf)x[d]; }
    qf cx = u[1] * v[2] - u[2] * v[1];
    qf cy = u[2] * v[0] - u[0] * v[2];
    qf cz = u[0] * v[1] - u[1] * v[0];
    g->area[k] = qsqrt(cx * cx + cy * cy + cz * cz) / 2;
  }
  return 1;
}

/* Local system of one element.
 *   C(T)[k][j] = sigma_k |F_k| / 3 if vertex j lies on F_k (Eq. C(T)); rows of
 *                Neumann faces carry no multiplier and are zero here;
 *   A = a K + c M;
 *   B_j = |T|/4 sum_k f(Ct_k) phi_j(Ct_k) + sum_{k Neumann} |F_k| g_k phi_j(Ct_k);
 *   S = C A^-1 C',  g = -C A^-1 B  (both n = 4 rows; zero rows for Neumann). */
typedef struct {
  qf A[4][4], C[4][4], B[4];
} local_q;

static int local_system(const double P[4][3], double a, double c, const double f4[4],
                        const int32_t sig4[4], const int32_t kind4[4], const double g4[4],
                        geom_q* G, local_q* L) {
  if (!geom(P, G)) return 0;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) L->A[i][j] = (qf)a * G->K[i][j] + (qf)c * G->M[i][j];
  for (int k = 0; k < 4; ++k)
    for (int j = 0; j < 4; ++j) {
      qf val = on_face(k, j) ? (qf)sig4[k] * G->area[k] / 3 : 0;
      L->C[k][j] = (kind4[k] == KIND_NEUMANN) ? 0 : val;
    }
  for (int j = 0; j < 4; ++j) {
    qf s = 0, ln = 0;
    for (int k = 0; k < 4; ++k)
      if (on_face(k, j)) {
        s += (qf)f4[k] / 3;
        if (kind4[k] == KIND_NEUMANN && g4) ln += G->area[k] * (qf)g4[k] / 3;
      }
    L->B[j] = G->vol / 4 * s + ln;
  }
  return 1;
}

/* Exported: S (4x4 row-major) and g (4) of one element, rounded to fp64. */
int or_tet_local(const double* P12, double a, double c, const double* f4, const int32_t* sig4,
                 const int32_t* kind4, const double* g4, double* S16, double* g_out) {
  double P[4][3];
  for (int i = 0; i < 4; ++i)
    for (int d = 0; d < 3; ++d) P[i][d] = P12[3 * i + d];
  geom_q G;
  local_q L;
  if (!local_system(P, a, c, f4, sig4, kind4, g4, &G, &L)) return OR_ERR_DEGENERATE;
  qf A[4][4], R[4][8];
  memcpy(A, L.A, sizeof A);
  for (int j = 0; j < 4; ++j) {
    for (int k = 0; k < 4; ++k) R[j][k] = L.C[k][j]; /* C' */
    R[j][4] = L.B[j];
  }
  if (!qsolve(4, A, 5, R)) return OR_ERR_DEGENERATE;
  for (int k = 0; k < 4; ++k) {
    for (int m = 0; m < 4; ++m) {
      qf s = 0;
      for (int j = 0; j < 4; ++j) s += L.C[k][j] * R[j][m];
      S16[4 * k + m] = (double)s;
    }
    qf s = 0;
    for (int j = 0; j < 4; ++j) s += L.C[k][j] * R[j][4];
    g_out[k] = (double)(-s);
  }
  return OR_OK;
}

/* Exported for checks against closed forms: K, M, C (all faces, given sigma),
 * areas, volume and B for one element, rounded to fp64. */
int or_tet_matrices(const double* P12, const double* f4, const int32_t* sig4, double* K16,
                    double* M16, double* C16, double* area4, double* vol, double* B4) {
  double P[4][3];
  for (int i = 0; i < 4; ++i)
    for (int d = 0; d < 3; ++d) P[i][d] = P12[3 * i + d];
  geom_q G;
  local_q L;
  int32_t kinds[4] = {0, 0, 0, 0};
  if (!local_system(P, 1.0, 1.0, f4, sig4, kinds, NULL, &G, &L)) return OR_ERR_DEGENERATE;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      K16[4 * i + j] = (double)G.K[i][j];
      M16[4 * i + j] = (double)G.M[i][j];
      C16[4 * i + j] = (double)L.C[i][j];
    }
  for (int k = 0; k < 4; ++k) { area4[k] = (double)G.area[k]; B4[k] = (double)L.B[k]; }
  *vol = (double)G.vol;
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Faces (Section 3.3 FacesUp semantics, plus the Neumann list of Listing 1)  */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t v[3];
  int64_t slot; /* 4t+k for tet faces, 4nE+i for the i-th Neumann triple */
} rec_t;

static int cmp_rec(const void* pa, const void* pb) {
  const rec_t* a = (const rec_t*)pa;
  const rec_t* b = (const rec_t*)pb;
  for (int i = 0; i < 3; ++i)
    if (a->v[i] != b->v[i]) return a->v[i] < b->v[i] ? -1 : 1;
  return (a->slot > b->slot) - (a->slot < b->slot);
}

static void sort3(int32_t v[3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j)
      if (v[j] < v[i]) { int32_t t = v[i]; v[i] = v[j]; v[j] = t; }
}

/* tet_face[4nE]: face id, bit 31 set when sigma = -1 (second occurrence).
 * face_tet[2 nF]: T+, T- (-1 if boundary).  face_vtx[3 nF]: T+'s local tuple.
 * face_kind[nF]: interior / Dirichlet / Neumann.  Output arrays must hold the
 * upper bound nF <= 4 nE. */
int or_faces(int64_t nE, int64_t nC, const int32_t* tet, int64_t nN, const int32_t* nb,
             int32_t* tet_face, int32_t* face_tet, int32_t* face_vtx, int8_t* face_kind,
             int64_t* nF_out) {
  *nF_out = 0;
  if (nE < 0 || nC < 0 || nN < 0) return OR_ERR_ARG;
  if (4 * nE + nN >= ((int64_t)1 << 31)) return OR_ERR_OVERFLOW;
  for (int64_t t = 0; t < nE; ++t)
    for (int i = 0; i < 4; ++i) {
      if (tet[4 * t + i] < 0 || tet[4 * t + i] >= nC) return OR_ERR_ARG;
      for (int j = 0; j < i; ++j)
        if (tet[4 * t + i] == tet[4 * t + j]) return OR_ERR_ARG;
    }
  for (int64_t i = 0; i < nN; ++i)
    for (int j = 0; j < 3; ++j) {
      if (nb[3 * i + j] < 0 || nb[3 * i + j] >= nC) return OR_ERR_ARG;
      for (int l = 0; l < j; ++l)
        if (nb[3 * i + j] == nb[3 * i + l]) return OR_ERR_ARG;
    }
  int64_t nrec = 4 * nE + nN;
  rec_t* rec = (rec_t*)malloc(sizeof(rec_t) * (size_t)(nrec > 0 ? nrec : 1));
  int64_t* mate = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nE > 0 ? 4 * nE : 1));
  char* first = (char*)calloc((size_t)(nE > 0 ? 4 * nE : 1), 1);
  char* neu = (char*)calloc((size_t)(nE > 0 ? 4 * nE : 1), 1);
  if (!rec || !mate || !first || !neu) {
    free(rec); free(mate); free(first); free(neu);
    return OR_ERR_NOMEM;
  }
  for (int64_t t = 0; t < nE; ++t)
    for (int k = 0; k < 4; ++k) {
      rec_t* r = &rec[4 * t + k];
      for (int j = 0; j < 3; ++j) r->v[j] = tet[4 * t + LFACE[k][j]];
      sort3(r->v);
      r->slot = 4 * t + k;
    }
  for (int64_t i = 0; i < nN; ++i) {
    rec_t* r = &rec[4 * nE + i];
    for (int j = 0; j < 3; ++j) r->v[j] = nb[3 * i + j];
    sort3(r->v);
    r->slot = 4 * nE + i;
  }
  qsort(rec, (size_t)nrec, sizeof(rec_t), cmp_rec);
  int status = OR_OK;
  for (int64_t s = 0; s < 4 * nE; ++s) mate[s] = -1;
  for (int64_t i = 0; i < nrec && status == OR_OK;) {
    int64_t j = i;
    while (j < nrec && rec[j].v[0] == rec[i].v[0] && rec[j].v[1] == rec[i].v[1] &&
           rec[j].v[2] == rec[i].v[2])
      ++j;
    int64_t nt = 0, nn = 0, s0 = -1, s1 = -1;
    for (int64_t l = i; l < j; ++l) {
      if (rec[l].slot < 4 * nE) {
        if (nt == 0) s0 = rec[l].slot; else if (nt == 1) s1 = rec[l].slot;
        ++nt;
      } else {
        ++nn;
      }
    }
    if (nt > 2) status = OR_ERR_NONMANIFOLD;
    else if (nt == 0 || nn > 1 || (nt == 2 && nn > 0)) status = OR_ERR_ARG;
    else {
      first[s0] = 1;
      neu[s0] = (char)(nn > 0);
      if (nt == 2) { mate[s0] = s1; mate[s1] = s0; }
    }
    i = j;
  }
  if (status == OR_OK) {
    int64_t nF = 0;
    for (int64_t s = 0; s < 4 * nE; ++s) {
      if (first[s]) {
        int64_t id = nF++;
        int64_t t = s / 4;
        int k = (int)(s % 4);
        tet_face[s] = (int32_t)id;
        face_tet[2 * id] = (int32_t)t;
        face_tet[2 * id + 1] = mate[s] >= 0 ? (int32_t)(mate[s] / 4) : -1;
        for (int j = 0; j < 3; ++j) face_vtx[3 * id + j] = tet[4 * t + LFACE[k][j]];
        face_kind[id] = (int8_t)(mate[s] >= 0 ? KIND_INTERIOR : (neu[s] ? KIND_NEUMANN : KIND_DIRICHLET));
      } else {
        /* the first occurrence of this face has a smaller slot: already numbered */
        tet_face[s] = (int32_t)((uint32_t)tet_face[mate[s]] | 0x80000000u);
      }
    }
    *nF_out = nF;
  }
  free(rec); free(mate); free(first); free(neu);
  return status;
}

/* Multiplier numbering: l(F) = rank of F among non-Neumann faces in face order
 * (the RFaces restriction of Listing SchurComplement_vectorization). */
int or_multipliers(int64_t nF, const int8_t* face_kind, int32_t* face_mult, int64_t* L_out) {
  int64_t L = 0;
  for (int64_t F = 0; F < nF; ++F) face_mult[F] = face_kind[F] == KIND_NEUMANN ? -1 : (int32_t)L++;
  *L_out = L;
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* CSR pattern of sum_T P_T' S(T) P_T: (l(F_k), l(F_m)) for all non-Neumann   */
/* k, m of every tet, columns sorted, duplicates merged.                      */
/* ------------------------------------------------------------------------ */
typedef struct { int32_t r, c; } pair_t;
static int cmp_pair(const void* pa, const void* pb) {
  const pair_t* a = (const pair_t*)pa;
  const pair_t* b = (const pair_t*)pb;
  if (a->r != b->r) return a->r < b->r ? -1 : 1;
  return (a->c > b->c) - (a->c < b->c);
}

int or_csr_pattern(int64_t nE, const int32_t* tet_face, const int32_t* face_mult, int64_t L,
                   int32_t* rowptr, int32_t* colind, int64_t* nnz_out) {
  pair_t* p = (pair_t*)malloc(sizeof(pair_t) * (size_t)(nE > 0 ? 16 * nE : 1));
  if (!p) return OR_ERR_NOMEM;
  int64_t np_ = 0;
  for (int64_t t = 0; t < nE; ++t)
    for (int k = 0; k < 4; ++k) {
      int32_t lk = face_mult[tet_face[4 * t + k] & 0x7fffffff];
      if (lk < 0) continue;
      for (int m = 0; m < 4; ++m) {
        int32_t lm = face_mult[tet_face[4 * t + m] & 0x7fffffff];
        if (lm < 0) continue;
        p[np_].r = lk;
        p[np_].c = lm;
        ++np_;
      }
    }
  qsort(p, (size_t)np_, sizeof(pair_t), cmp_pair);
  int64_t nnz = 0;
  for (int64_t i = 0; i <= L; ++i) rowptr[i] = 0;
  for (int64_t i = 0; i < np_; ++i) {
    if (i > 0 && p[i].r == p[i - 1].r && p[i].c == p[i - 1].c) continue;
    if (nnz >= ((int64_t)1 << 31) - 1) { free(p); return OR_ERR_OVERFLOW; }
    colind[nnz++] = p[i].c;
    rowptr[p[i].r + 1]++;
  }
  for (int64_t i = 0; i < L; ++i) rowptr[i + 1] += rowptr[i];
  *nnz_out = nnz;
  free(p);
  return OR_OK;
}

/* centroid of face tuple [x y z]: (P_x + P_y + P_z)/3 (Listing StiffMassPH) */
int or_face_centroids(int64_t nF, const int32_t* face_vtx, const double* coord, double* out) {
  for (int64_t F = 0; F < nF; ++F)
    for (int d = 0; d < 3; ++d)
      out[3 * F + d] = (coord[3 * (int64_t)face_vtx[3 * F] + d] + coord[3 * (int64_t)face_vtx[3 * F + 1] + d] +
                        coord[3 * (int64_t)face_vtx[3 * F + 2] + d]) / 3.0;
  return OR_OK;
}

static void gather_tet(const double* coord, const int32_t* tet, int64_t t, double P[4][3]) {
  for (int i = 0; i < 4; ++i)
    for (int d = 0; d < 3; ++d) P[i][d] = coord[3 * (int64_t)tet[4 * t + i] + d];
}

static int64_t find_col(const int32_t* rowptr, const int32_t* colind, int32_t row, int32_t col) {
  int64_t lo = rowptr[row], hi = rowptr[row + 1] - 1;
  while (lo <= hi) {
    int64_t mid = (lo + hi) / 2;
    if (colind[mid] == col) return mid;
    if (colind[mid] < col) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

static int add_dirichlet(int64_t nF, const double* coord, const int8_t* face_kind, const int32_t* face_mult,
                         const int32_t* face_vtx, const double* uD_face, double* rhs, double* rhs_abs);

/* H[l(F_k), l(F_m)] += S[k][m] and rhs[l(F_k)] += g[k] for the non-Neumann
 * local faces of one element (P_T' S(T) P_T in Algorithm 1's assembly). */
static int scatter_element(const int32_t mult[4], const double S[16], const double g[4], const int32_t* rowptr,
                           const int32_t* colind, double* values, double* rhs, double* rhs_abs) {
  for (int k = 0; k < 4; ++k) {
    if (mult[k] < 0) continue;
    for (int m = 0; m < 4; ++m) {
      if (mult[m] < 0) continue;
      int64_t pos = find_col(rowptr, colind, mult[k], mult[m]);
      if (pos < 0) return OR_ERR_ARG;
      values[pos] += S[4 * k + m];
    }
    rhs[mult[k]] += g[k];
    rhs_abs[mult[k]] += fabs(g[k]);
  }
  return OR_OK;
}

/* Inputs of element t: vertices, and per local face sigma, kind, multiplier,
 * f and g. */
static void element_inputs(int64_t t, const double* coord, const int32_t* tet, const int32_t* tet_face,
                           const int8_t* face_kind, const int32_t* face_mult, const double* f_face,
                           const double* gN_face, double P[4][3], int32_t sig[4], int32_t kind[4],
                           int32_t mult[4], double f4[4], double g4[4]) {
  gather_tet(coord, tet, t, P);
  for (int k = 0; k < 4; ++k) {
    int32_t tf = tet_face[4 * t + k];
    int32_t F = tf & 0x7fffffff;
    sig[k] = (tf < 0) ? -1 : 1;
    kind[k] = face_kind[F];
    mult[k] = face_mult[F];
    f4[k] = f_face[F];
    g4[k] = gN_face ? gN_face[F] : 0.0;
  }
}

/* S(T) and g(T) of element t (Eq. schur, Algorithm 1 first loop) and the
 * multiplier ids of its faces. */
static int condense_element(int64_t t, const double* coord, const int32_t* tet, const int32_t* tet_face,
                            const int8_t* face_kind, const int32_t* face_mult, const double* a, double c,
                            const double* f_face, const double* gN_face, int32_t mult[4], double S[16],
                            double g[4]) {
  double P[4][3], f4[4], g4[4];
  int32_t sig[4], kind[4];
  element_inputs(t, coord, tet, tet_face, face_kind, face_mult, f_face, gN_face, P, sig, kind, mult, f4, g4);
  if (!(a[t] > 0) || !isfinite(a[t])) return OR_ERR_ARG;
  return or_tet_local(&P[0][0], a[t], c, f4, sig, kind, g4, S, g);
}

/* Global condensed system H Lambda = rhs with H = sum_T P_T' S(T) P_T and
 * rhs = sum_T P_T' g(T) + b_D, b_D(F) = |F| u_D(Ct_F) on Dirichlet faces
 * (Section 4.3).  values is aligned with (rowptr, colind).  rhs_abs receives the
 * sum of the magnitudes of the addends of each rhs entry (a scale for
 * comparisons, since interior contributions cancel). */
int or_assemble(int64_t nE, const double* coord, const int32_t* tet, const int32_t* tet_face,
                int64_t nF, const int8_t* face_kind, const int32_t* face_mult,
                const int32_t* face_vtx, int64_t L, const int32_t* rowptr, const int32_t* colind,
                const double* a, double c, const double* f_face, const double* uD_face,
                const double* gN_face, double* values, double* rhs, double* rhs_abs) {
  int64_t nnz = rowptr[L];
  for (int64_t i = 0; i < nnz; ++i) values[i] = 0;
  for (int64_t i = 0; i < L; ++i) { rhs[i] = 0; rhs_abs[i] = 0; }
  if (!(c > 0) || !isfinite(c)) return OR_ERR_ARG;
  for (int64_t t = 0; t < nE; ++t) {
    double S[16], g[4];
    int32_t mult[4];
    int st = condense_element(t, coord, tet, tet_face, face_kind, face_mult, a, c, f_face, gN_face, mult, S, g);
    if (st != OR_OK) return st;
    st = scatter_element(mult, S, g, rowptr, colind, values, rhs, rhs_abs);
    if (st != OR_OK) return st;
  }
  return add_dirichlet(nF, coord, face_kind, face_mult, face_vtx, uD_face, rhs, rhs_abs);
}

/* Element chunk of the multi-threaded loops below. */
#define OR_CHUNK ((int64_t)1 << 18)

/* or_assemble with the element computations shared out across `nthreads`
 * threads (OpenMP): each element's S(T), g(T) go to a buffer, and one thread
 * then scatters them in element order, so values and rhs are bit-identical to
 * or_assemble's.  The first error in element order is returned, as there. */
int or_assemble_mt(int64_t nE, const double* coord, const int32_t* tet, const int32_t* tet_face,
                   int64_t nF, const int8_t* face_kind, const int32_t* face_mult,
                   const int32_t* face_vtx, int64_t L, const int32_t* rowptr, const int32_t* colind,
                   const double* a, double c, const double* f_face, const double* uD_face,
                   const double* gN_face, double* values, double* rhs, double* rhs_abs, int nthreads) {
  int64_t nnz = rowptr[L];
  for (int64_t i = 0; i < nnz; ++i) values[i] = 0;
  for (int64_t i = 0; i < L; ++i) { rhs[i] = 0; rhs_abs[i] = 0; }
  if (!(c > 0) || !isfinite(c)) return OR_ERR_ARG;
  const int64_t cap = nE < OR_CHUNK ? (nE > 0 ? nE : 1) : OR_CHUNK;
  double* S = (double*)malloc(sizeof(double) * 16 * (size_t)cap);
  double* g = (double*)malloc(sizeof(double) * 4 * (size_t)cap);
  int32_t* mult = (int32_t*)malloc(sizeof(int32_t) * 4 * (size_t)cap);
  int* st = (int*)malloc(sizeof(int) * (size_t)cap);
  if (!S || !g || !mult || !st) {
    free(S); free(g); free(mult); free(st);
    return OR_ERR_NOMEM;
  }
  int status = OR_OK;
  for (int64_t t0 = 0; t0 < nE && status == OR_OK; t0 += OR_CHUNK) {
    const int64_t n = nE - t0 < OR_CHUNK ? nE - t0 : OR_CHUNK;
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads)
    for (int64_t i = 0; i < n; ++i)
      st[i] = condense_element(t0 + i, coord, tet, tet_face, face_kind, face_mult, a, c, f_face, gN_face,
                               mult + 4 * i, S + 16 * i, g + 4 * i);
    for (int64_t i = 0; i < n && status == OR_OK; ++i) {
      status = st[i];
      if (status == OR_OK)
        status = scatter_element(mult + 4 * i, S + 16 * i, g + 4 * i, rowptr, colind, values, rhs, rhs_abs);
    }
  }
  free(S); free(g); free(mult); free(st);
  if (status != OR_OK) return status;
  return add_dirichlet(nF, coord, face_kind, face_mult, face_vtx, uD_face, rhs, rhs_abs);
}

/* b_D(F) = |F| u_D(Ct_F), added once per Dirichlet face (Section 4.3). */
static int add_dirichlet(int64_t nF, const double* coord, const int8_t* face_kind, const int32_t* face_mult,
                         const int32_t* face_vtx, const double* uD_face, double* rhs, double* rhs_abs) {
  if (uD_face) {
    for (int64_t F = 0; F < nF; ++F) {
      if (face_kind[F] != KIND_DIRICHLET) continue;
      qf u[3], v[3];
      const double* x = &coord[3 * (int64_t)face_vtx[3 * F]];
      const double* y = &coord[3 * (int64_t)face_vtx[3 * F + 1]];
      const double* z = &coord[3 * (int64_t)face_vtx[3 * F + 2]];
      for (int d = 0; d < 3; ++d) { u[d] = (qf)z[d] - (qf)x[d]; v[d] = (qf)y[d] - (qf)x[d]; }
      qf cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
      double bD = (double)(qsqrt(cx * cx + cy * cy + cz * cz) / 2 * (qf)uD_face[F]);
      rhs[face_mult[F]] += bD;
      rhs_abs[face_mult[F]] += fabs(bD);
    }
  }
  return OR_OK;
}

/* Recovery of element t: U(T) = A^-1 (B + C' Lambda_T) into U[4t..4t+3]. */
static int recover_element(int64_t t, const double* coord, const int32_t* tet, const int32_t* tet_face,
                           const int8_t* face_kind, const int32_t* face_mult, const double* a, double c,
                           const double* f_face, const double* gN_face, const double* lambda, double* U) {
  double P[4][3], f4[4], g4[4];
  int32_t sig[4], kind[4], mult[4];
  qf lam[4];
  element_inputs(t, coord, tet, tet_face, face_kind, face_mult, f_face, gN_face, P, sig, kind, mult, f4, g4);
  for (int k = 0; k < 4; ++k) lam[k] = mult[k] >= 0 ? (qf)lambda[mult[k]] : 0;
  if (!(a[t] > 0) || !isfinite(a[t])) return OR_ERR_ARG;
  geom_q G;
  local_q Lq;
  if (!local_system(P, a[t], c, f4, sig, kind, g4, &G, &Lq)) return OR_ERR_DEGENERATE;
  qf A[4][4], R[4][8];
  memcpy(A, Lq.A, sizeof A);
  for (int j = 0; j < 4; ++j) {
    qf s = Lq.B[j];
    for (int k = 0; k < 4; ++k) s += Lq.C[k][j] * lam[k];
    R[j][0] = s;
  }
  if (!qsolve(4, A, 1, R)) return OR_ERR_DEGENERATE;
  for (int j = 0; j < 4; ++j) U[4 * t + j] = (double)R[j][0];
  return OR_OK;
}

/* Element recovery U(T) = A^-1 (B + C' Lambda_T), Lambda_T(k) = lambda[l(F_k)]
 * and 0 on Neumann faces (Algorithm 1, second loop). U is nE x 4. */
int or_recover(int64_t nE, const double* coord, const int32_t* tet, const int32_t* tet_face,
               const int8_t* face_kind, const int32_t* face_mult, const double* a, double c,
               const double* f_face, const double* gN_face, const double* lambda, double* U) {
  if (!(c > 0) || !isfinite(c)) return OR_ERR_ARG;
  for (int64_t t = 0; t < nE; ++t) {
    int st = recover_element(t, coord, tet, tet_face, face_kind, face_mult, a, c, f_face, gN_face, lambda, U);
    if (st != OR_OK) return st;
  }
  return OR_OK;
}

/* or_recover with the elements shared out across `nthreads` threads (OpenMP);
 * every element writes its own row of U, so U is bit-identical to
 * or_recover's.  The first error in element order is returned. */
int or_recover_mt(int64_t nE, const double* coord, const int32_t* tet, const int32_t* tet_face,
                  const int8_t* face_kind, const int32_t* face_mult, const double* a, double c,
                  const double* f_face, const double* gN_face, const double* lambda, double* U, int nthreads) {
  if (!(c > 0) || !isfinite(c)) return OR_ERR_ARG;
  int status = OR_OK;
  int64_t first_bad = nE;
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads)
  for (int64_t t = 0; t < nE; ++t) {
    int st = recover_element(t, coord, tet, tet_face, face_kind, face_mult, a, c, f_face, gN_face, lambda, U);
    if (st != OR_OK) {
#pragma omp critical
      if (t < first_bad) { first_bad = t; status = st; }
    }
  }
  return status;
}

/* Per-element local data for the monolithic check (Eq. VectorForm): A (4x4),
 * C rows (4x4, zero rows for Neumann faces) and B (4) of element t. */
int or_element_blocks(int64_t t, const double* coord, const int32_t* tet, const int32_t* tet_face,
                      const int8_t* face_kind, const double* a, double c, const double* f_face,
                      const double* gN_face, double* A16, double* C16, double* B4) {
  double P[4][3], f4[4], g4[4];
  int32_t sig[4], kind[4];
  gather_tet(coord, tet, t, P);
  for (int k = 0; k < 4; ++k) {
    int32_t tf = tet_face[4 * t + k];
    int32_t F = tf & 0x7fffffff;
    sig[k] = (tf < 0) ? -1 : 1;
    kind[k] = face_kind[F];
    f4[k] = f_face[F];
    g4[k] = gN_face ? gN_face[F] : 0.0;
  }
  geom_q G;
  local_q Lq;
  if (!local_system(P, a[t], c, f4, sig, kind, g4, &G, &Lq)) return OR_ERR_DEGENERATE;
  for (int i = 0; i < 4; ++i) {
    for (int j = 0; j < 4; ++j) { A16[4 * i + j] = (double)Lq.A[i][j]; C16[4 * i + j] = (double)Lq.C[i][j]; }
    B4[i] = (double)Lq.B[i];
  }
  return OR_OK;
}

/* Recovery of one element (Algorithm 1 second loop): U = A^-1 (B + C' lam4),
 * lam4[k] the multiplier of local face k (ignored on Neumann faces). */
int or_tet_recover(const double* P12, double a, double c, const double* f4, const int32_t* sig4,
                   const int32_t* kind4, const double* g4, const double* lam4, double* U4) {
  double P[4][3];
  for (int i = 0; i < 4; ++i)
    for (int d = 0; d < 3; ++d) P[i][d] = P12[3 * i + d];
  geom_q G;
  local_q Lq;
  if (!local_system(P, a, c, f4, sig4, kind4, g4, &G, &Lq)) return OR_ERR_DEGENERATE;
  qf A[4][4], R[4][8];
  memcpy(A, Lq.A, sizeof A);
  for (int j = 0; j < 4; ++j) {
    qf s = Lq.B[j];
    for (int k = 0; k < 4; ++k)
      if (kind4[k] != KIND_NEUMANN) s += Lq.C[k][j] * (qf)lam4[k];
    R[j][0] = s;
  }
  if (!qsolve(4, A, 1, R)) return OR_ERR_DEGENERATE;
  for (int j = 0; j < 4; ++j) U4[j] = (double)R[j][0];
  return OR_OK;
}

/* r = b - H x for a CSR matrix H (rowptr [n+1], colind, values), with each
 * row's sum formed in binary128 and rounded once: the residual of iterative
 * refinement, accurate beyond what an fp64 sum gives when H is ill
 * conditioned (Eq. schur's system solved to fp64 accuracy). */
int or_residual(int64_t n, const int32_t* rowptr, const int32_t* colind, const double* values, const double* x,
                const double* b, double* r) {
  for (int64_t i = 0; i < n; ++i) {
    qf s = (qf)b[i];
    for (int32_t j = rowptr[i]; j < rowptr[i + 1]; ++j) s -= (qf)values[j] * (qf)x[colind[j]];
    r[i] = (double)s;
  }
  return OR_OK;
}
