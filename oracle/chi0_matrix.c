/*
 * Oracle: chi0_{mu nu}(R, tau) from the four-term matrix form of Sec. 2 (the equation obtained
 * by combining Eqs. chi0_NAOs, chi0_ABFs and LRI), evaluated term by term in plain C.
 * TEST INFRASTRUCTURE ONLY: compiled into the oracle's own shared library and called by tests
 * and by the CPU-baseline leg of the benchmark; the GPU library never links it.
 *
 * In the real convention (oracle package docstring: G(i tau) -> G^vir, G(-i tau) -> G^occ, the
 * complex conjugates of the second and fourth lines swapping the two) the four lines read, for
 * mu on atom U in the home cell and nu on atom V in cell R,
 *
 *   line 1:  sum_{K(R1)} sum_{ik} C^mu_{i, k(R1)} sum_j G^vir_{ij}(R) sum_{L(R2)} sum_l C^nu_{j, l(R2-R)} G^occ_{lk}(R1-R2)
 *   line 2:  the same with G^vir and G^occ exchanged
 *   line 3:  sum_{K(R1)} sum_{ik} C^mu_{i, k(R1)} sum_j G^occ_{jk}(R1-R) sum_{L(R2)} sum_l C^nu_{j, l(R2-R)} G^vir_{il}(R2)
 *   line 4:  the same with G^vir and G^occ exchanged
 *
 * and chi0(R, tau) = -s (line 1 + line 2 + line 3 + line 4), s the spin factor.  The sums are
 * taken here in this order, with intermediates of this file's own:
 *
 *   lines 1, 2 (for each neighbour K(R1) of U; A, B = the line's first and second G):
 *     P^mu_{jk} = sum_i C^mu_{i,k(R1)} A_{ij}(R)                       (the U side first)
 *     Q^nu_{jk} = sum_{L(R2)} sum_l C^nu_{j,l(R2-R)} B_{lk}(R1 - R2)    (the V side)
 *     line     += sum_{jk} P^mu_{jk} Q^nu_{jk}
 *   lines 3, 4 (the sum over K(R1) and the one over L(R2) separate; A, B as above):
 *     F^mu_{ij} = sum_{K(R1)} sum_k C^mu_{i,k(R1)} A_{jk}(R1 - R)
 *     H^nu_{ij} = sum_{L(R2)} sum_l C^nu_{j,l(R2-R)} B_{il}(R2)
 *     line      = sum_{ij} F^mu_{ij} H^nu_{ij}
 *
 * Stored LRI blocks: C[I, K, R][mu][i][k] = C^{mu(0)}_{i(0), k(R)} (mu, i on atom I in the home
 * cell, k on atom K in cell R).  A neighbour L(R2) of V(R) is a stored block C[V, L, R2 - R].
 * G arrays are [ntau][nR][nao][nao] on the BvK mesh; a lattice vector is folded into the mesh
 * before indexing.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int natoms, nao, naux, nk1, nk2, nk3, nR;
  const int *n_ao, *n_aux, *ao_off, *aux_off;
  int nblk;
  const int *blk_I, *blk_K, *blk_R;   /* blk_R[3*b + 0..2] */
  const long *blk_off;                /* offset of block b in C */
  const double *C;
  int *first, *order;                 /* blocks with atom a first: order[first[a] .. first[a+1]-1] */
} sys_t;

static int fold(int x, int n) { int r = x % n; return r < 0 ? r + n : r; }

static int bvk(const sys_t *s, int r0, int r1, int r2) {
  return (fold(r0, s->nk1) * s->nk2 + fold(r1, s->nk2)) * s->nk3 + fold(r2, s->nk3);
}

/* element (a, b) of G(R) with a an NAO of atom A and b one of atom B */
static double gab(const sys_t *s, const double *G, int iR, int A, int a, int B, int b) {
  return G[((long)iR * s->nao + s->ao_off[A] + a) * s->nao + s->ao_off[B] + b];
}

static void index_blocks(sys_t *s) {
  s->first = (int *)calloc((size_t)s->natoms + 1, sizeof(int));
  s->order = (int *)malloc(sizeof(int) * (size_t)(s->nblk > 0 ? s->nblk : 1));
  int *fill = (int *)calloc((size_t)s->natoms, sizeof(int));
  for (int b = 0; b < s->nblk; ++b) s->first[s->blk_I[b] + 1]++;
  for (int a = 0; a < s->natoms; ++a) s->first[a + 1] += s->first[a];
  for (int b = 0; b < s->nblk; ++b) s->order[s->first[s->blk_I[b]] + fill[s->blk_I[b]]++] = b;
  free(fill);
}

/* lines 1 and 2 for the pair (U, V(R)): adds sum over K(R1) of P:Q into acc[mu][nu] */
static void lines_12(const sys_t *s, int U, int V, const int Rv[3], int iR, const double *A, const double *B,
                     double *acc) {
  const int nU = s->n_ao[U], nV = s->n_ao[V], xU = s->n_aux[U], xV = s->n_aux[V];
  for (int t = s->first[U]; t < s->first[U + 1]; ++t) {
    const int bK = s->order[t], K = s->blk_K[bK], nK = s->n_ao[K];
    const int *R1 = s->blk_R + 3 * bK;
    const double *CU = s->C + s->blk_off[bK];   /* C^mu_{i, k(R1)}: [xU][nU][nK] */
    double *P = (double *)calloc((size_t)xU * nV * nK, sizeof(double));
    double *Q = (double *)calloc((size_t)xV * nV * nK, sizeof(double));
    for (int mu = 0; mu < xU; ++mu)
      for (int j = 0; j < nV; ++j)
        for (int k = 0; k < nK; ++k) {
          double p = 0.0;
          for (int i = 0; i < nU; ++i) p += CU[((long)mu * nU + i) * nK + k] * gab(s, A, iR, U, i, V, j);
          P[((long)mu * nV + j) * nK + k] = p;
        }
    for (int u = s->first[V]; u < s->first[V + 1]; ++u) {
      const int bL = s->order[u], L = s->blk_K[bL], nL = s->n_ao[L];
      const int *Rr = s->blk_R + 3 * bL;   /* R2 - R */
      const int iRlk = bvk(s, R1[0] - Rv[0] - Rr[0], R1[1] - Rv[1] - Rr[1], R1[2] - Rv[2] - Rr[2]);
      const double *CV = s->C + s->blk_off[bL];   /* C^nu_{j, l(R2-R)}: [xV][nV][nL] */
      for (int nu = 0; nu < xV; ++nu)
        for (int j = 0; j < nV; ++j)
          for (int k = 0; k < nK; ++k) {
            double q = 0.0;
            for (int l = 0; l < nL; ++l) q += CV[((long)nu * nV + j) * nL + l] * gab(s, B, iRlk, L, l, K, k);
            Q[((long)nu * nV + j) * nK + k] += q;
          }
    }
    const long jk = (long)nV * nK;
    for (int mu = 0; mu < xU; ++mu)
      for (int nu = 0; nu < xV; ++nu) {
        double d = 0.0;
        for (long e = 0; e < jk; ++e) d += P[mu * jk + e] * Q[nu * jk + e];
        acc[(long)mu * xV + nu] += d;
      }
    free(P);
    free(Q);
  }
}

/* lines 3 and 4 for the pair (U, V(R)): adds F:H into acc[mu][nu] */
static void lines_34(const sys_t *s, int U, int V, const int Rv[3], const double *A, const double *B,
                     double *acc) {
  const int nU = s->n_ao[U], nV = s->n_ao[V], xU = s->n_aux[U], xV = s->n_aux[V];
  const long ij = (long)nU * nV;
  double *F = (double *)calloc((size_t)xU * ij, sizeof(double));
  double *H = (double *)calloc((size_t)xV * ij, sizeof(double));
  for (int t = s->first[U]; t < s->first[U + 1]; ++t) {
    const int bK = s->order[t], K = s->blk_K[bK], nK = s->n_ao[K];
    const int *R1 = s->blk_R + 3 * bK;
    const int iRjk = bvk(s, R1[0] - Rv[0], R1[1] - Rv[1], R1[2] - Rv[2]);
    const double *CU = s->C + s->blk_off[bK];
    for (int mu = 0; mu < xU; ++mu)
      for (int i = 0; i < nU; ++i)
        for (int j = 0; j < nV; ++j) {
          double f = 0.0;
          for (int k = 0; k < nK; ++k) f += CU[((long)mu * nU + i) * nK + k] * gab(s, A, iRjk, V, j, K, k);
          F[mu * ij + (long)i * nV + j] += f;
        }
  }
  for (int u = s->first[V]; u < s->first[V + 1]; ++u) {
    const int bL = s->order[u], L = s->blk_K[bL], nL = s->n_ao[L];
    const int *Rr = s->blk_R + 3 * bL;
    const int iRil = bvk(s, Rv[0] + Rr[0], Rv[1] + Rr[1], Rv[2] + Rr[2]);   /* R2 = R + (R2 - R) */
    const double *CV = s->C + s->blk_off[bL];
    for (int nu = 0; nu < xV; ++nu)
      for (int i = 0; i < nU; ++i)
        for (int j = 0; j < nV; ++j) {
          double h = 0.0;
          for (int l = 0; l < nL; ++l) h += CV[((long)nu * nV + j) * nL + l] * gab(s, B, iRil, U, i, L, l);
          H[nu * ij + (long)i * nV + j] += h;
        }
  }
  for (int mu = 0; mu < xU; ++mu)
    for (int nu = 0; nu < xV; ++nu) {
      double d = 0.0;
      for (long e = 0; e < ij; ++e) d += F[mu * ij + e] * H[nu * ij + e];
      acc[(long)mu * xV + nu] += d;
    }
  free(F);
  free(H);
}

/*
 * chi0(R, tau) = -spin * (line 1 + line 2 + line 3 + line 4) for the requested points.
 *   pts[2*p + 0] = BvK index of R, pts[2*p + 1] = tau index;
 *   pairs: npairs (U, V) pairs, or npairs = 0 for all;
 *   out: [npts][naux][naux], only the requested blocks are written (others untouched).
 */
int oracle_chi0_matrix(int natoms, const int *n_ao, const int *n_aux, const int *kmesh, int nblk,
                       const int *blk_I, const int *blk_K, const int *blk_R, const long *blk_off,
                       const double *C, int ntau, const double *Go, const double *Gv, double spin,
                       int npts, const int *pts, int npairs, const int *pairs, double *out) {
  sys_t s;
  memset(&s, 0, sizeof(s));
  s.natoms = natoms;
  s.n_ao = n_ao;
  s.n_aux = n_aux;
  s.nk1 = kmesh[0];
  s.nk2 = kmesh[1];
  s.nk3 = kmesh[2];
  s.nR = kmesh[0] * kmesh[1] * kmesh[2];
  int *ao_off = (int *)malloc(sizeof(int) * (size_t)(natoms + 1));
  int *aux_off = (int *)malloc(sizeof(int) * (size_t)(natoms + 1));
  ao_off[0] = aux_off[0] = 0;
  for (int a = 0; a < natoms; ++a) {
    ao_off[a + 1] = ao_off[a] + n_ao[a];
    aux_off[a + 1] = aux_off[a] + n_aux[a];
  }
  s.ao_off = ao_off;
  s.aux_off = aux_off;
  s.nao = ao_off[natoms];
  s.naux = aux_off[natoms];
  s.nblk = nblk;
  s.blk_I = blk_I;
  s.blk_K = blk_K;
  s.blk_R = blk_R;
  s.blk_off = blk_off;
  s.C = C;
  index_blocks(&s);
  const long gstride = (long)s.nR * s.nao * s.nao;
  const int np = npairs > 0 ? npairs : natoms * natoms;
  const long nwork = (long)npts * np;
#pragma omp parallel for schedule(dynamic, 1)
  for (long w = 0; w < nwork; ++w) {
    const int p = (int)(w / np), q = (int)(w % np);
    const int U = npairs > 0 ? pairs[2 * q] : q / natoms;
    const int V = npairs > 0 ? pairs[2 * q + 1] : q % natoms;
    const int iR = pts[2 * p], it = pts[2 * p + 1];
    if (it < 0 || it >= ntau || iR < 0 || iR >= s.nR) continue;
    const int Rv[3] = {iR / (s.nk2 * s.nk3), (iR / s.nk3) % s.nk2, iR % s.nk3};
    const double *gv = Gv + it * gstride, *go = Go + it * gstride;
    double *acc = (double *)calloc((size_t)n_aux[U] * n_aux[V], sizeof(double));
    lines_12(&s, U, V, Rv, iR, gv, go, acc);   /* line 1: G^vir(R) with G^occ(R1 - R2) */
    lines_12(&s, U, V, Rv, iR, go, gv, acc);   /* line 2: exchanged */
    lines_34(&s, U, V, Rv, go, gv, acc);       /* line 3: G^occ(R1 - R) with G^vir(R2) */
    lines_34(&s, U, V, Rv, gv, go, acc);       /* line 4: exchanged */
    double *dst = out + (long)p * s.naux * s.naux;
    for (int mu = 0; mu < n_aux[U]; ++mu)
      for (int nu = 0; nu < n_aux[V]; ++nu)
        dst[(long)(aux_off[U] + mu) * s.naux + aux_off[V] + nu] = -spin * acc[(long)mu * n_aux[V] + nu];
    free(acc);
  }
  free(s.first);
  free(s.order);
  free(ao_off);
  free(aux_off);
  return 0;
}
