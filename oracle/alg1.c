/*
 * Oracle: Algorithm 1 of the paper (loop structure evaluating chi0_{mu nu}(R, i tau)),
 * written out loop by loop in plain C.  TEST INFRASTRUCTURE ONLY: this file is
 * compiled into the oracle's own shared library and is called by tests and by the
 * CPU-baseline leg of the benchmark; the GPU library never links it.
 *
 * For every (R, tau) and every atom pair <U(0), V(R)>:
 *   X^nu_{ij}(R)       = sum_{L(R2) in N[V(R)]} sum_l C^{nu(0)}_{j(0), l(R2-R)} G_{il}(R2, i tau)
 *   for every K(R1) in N[U(0)]:
 *     N^nu_{jk}(R1, R) = sum_{L(R2) in N[V(R)]} sum_l C^{nu(0)}_{j(0), l(R2-R)} G_{lk}(R1-R2, -i tau)
 *     M^nu_{ik}        = sum_{j in V} G_{ij}(R, i tau) N^nu_{jk}
 *     Z^nu_{ik}        = sum_{j in V} G_{jk}(R1-R, -i tau) X^nu_{ij}
 *     O^nu_{ik}        = M + M*(-i tau) + Z + Z*(-i tau)
 *     chi0_{mu nu}    += sum_{i k} C^{mu(0)}_{i(0), k(R1)} O^nu_{ik}
 *
 * Real convention (see the oracle package docstring): the paper's G(i tau) is
 * +i G^vir(tau) and G(-i tau) is -i G^occ(tau); every product above pairs one of
 * each, so M = G^vir N[G^occ], M*(-i tau) = G^occ N[G^vir], Z = G^occ X[G^vir],
 * Z*(-i tau) = G^vir X[G^occ], all real, and chi0(tau) = -s * sum C O.
 *
 * Stored LRI blocks: C[I, K, R][mu][i][k] = C^{mu(0)}_{i(0), k(R)} (mu, i on atom I
 * in the home cell, k on atom K in cell R).  A neighbour L(R2) of V(R) is a stored
 * block C[V, L, R2 - R].  G arrays are [ntau][nR][nao][nao] on the BvK mesh, so a
 * lattice vector is folded into the mesh before indexing.
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
  /* per-atom list of blocks with that atom first: first[a] .. first[a+1]-1 in order[] */
  int *first, *order;
} sys_t;

static int fold(int x, int n) { int r = x % n; return r < 0 ? r + n : r; }

static int bvk(const sys_t *s, int r0, int r1, int r2) {
  return (fold(r0, s->nk1) * s->nk2 + fold(r1, s->nk2)) * s->nk3 + fold(r2, s->nk3);
}

/* G_{ij}(R) for atoms (A, B): element (i, j) of the block */
static double gel(const sys_t *s, const double *G, int iR, int A, int i, int B, int j) {
  return G[((long)iR * s->nao + s->ao_off[A] + i) * s->nao + s->ao_off[B] + j];
}

static void build_lists(sys_t *s) {
  s->first = (int *)calloc((size_t)s->natoms + 1, sizeof(int));
  s->order = (int *)malloc(sizeof(int) * (size_t)(s->nblk > 0 ? s->nblk : 1));
  for (int b = 0; b < s->nblk; ++b) s->first[s->blk_I[b] + 1]++;
  for (int a = 0; a < s->natoms; ++a) s->first[a + 1] += s->first[a];
  int *fill = (int *)calloc((size_t)s->natoms, sizeof(int));
  for (int b = 0; b < s->nblk; ++b) {
    int a = s->blk_I[b];
    s->order[s->first[a] + fill[a]++] = b;
  }
  free(fill);
}

/* One (U, V, R, tau) block of chi0 (un-scaled sum C O), added into out[mu][nu] (ld = ldo). */
static void pair_block(const sys_t *s, int U, int V, const int Rv[3], int iR,
                       const double *Ga /* G^vir(tau) */, const double *Gb /* G^occ(tau) */,
                       double *out, int ldo) {
  const int nU = s->n_ao[U], nV = s->n_ao[V], nauxU = s->n_aux[U], nauxV = s->n_aux[V];
  /* X for both Green's functions: X[g][nu][i][j], g = 0 uses G^vir, g = 1 uses G^occ */
  double *X = (double *)calloc((size_t)2 * nauxV * nU * nV, sizeof(double));
  for (int g = 0; g < 2; ++g) {
    const double *G = g == 0 ? Ga : Gb;
    for (int t = s->first[V]; t < s->first[V + 1]; ++t) {
      int b = s->order[t];
      int L = s->blk_K[b];
      const int *Rrel = s->blk_R + 3 * b;
      /* R2 = R + Rrel; G_{il}(R2) */
      int iR2 = bvk(s, Rv[0] + Rrel[0], Rv[1] + Rrel[1], Rv[2] + Rrel[2]);
      int nL = s->n_ao[L];
      const double *Cb = s->C + s->blk_off[b];
      for (int nu = 0; nu < nauxV; ++nu)
        for (int i = 0; i < nU; ++i)
          for (int j = 0; j < nV; ++j) {
            double acc = 0.0;
            for (int l = 0; l < nL; ++l)
              acc += Cb[((long)nu * nV + j) * nL + l] * gel(s, G, iR2, U, i, L, l);
            X[(((long)g * nauxV + nu) * nU + i) * nV + j] += acc;
          }
    }
  }
  for (int t1 = s->first[U]; t1 < s->first[U + 1]; ++t1) {
    int bK = s->order[t1];
    int K = s->blk_K[bK];
    const int *R1 = s->blk_R + 3 * bK;
    int nK = s->n_ao[K];
    const double *CU = s->C + s->blk_off[bK];
    /* N[g][nu][j][k]: g = 0 uses G(-i tau) = G^occ (paired with G^vir in M),
       g = 1 uses G^vir (the tau -> -tau partner) */
    double *N = (double *)calloc((size_t)2 * nauxV * nV * nK, sizeof(double));
    for (int g = 0; g < 2; ++g) {
      const double *G = g == 0 ? Gb : Ga;
      for (int t2 = s->first[V]; t2 < s->first[V + 1]; ++t2) {
        int bL = s->order[t2];
        int L = s->blk_K[bL];
        const int *Rrel = s->blk_R + 3 * bL;
        /* G_{lk}(R1 - R2) with R2 = R + Rrel */
        int iRlk = bvk(s, R1[0] - Rv[0] - Rrel[0], R1[1] - Rv[1] - Rrel[1], R1[2] - Rv[2] - Rrel[2]);
        int nL = s->n_ao[L];
        const double *CV = s->C + s->blk_off[bL];
        for (int nu = 0; nu < nauxV; ++nu)
          for (int j = 0; j < nV; ++j)
            for (int k = 0; k < nK; ++k) {
              double acc = 0.0;
              for (int l = 0; l < nL; ++l)
                acc += CV[((long)nu * nV + j) * nL + l] * gel(s, G, iRlk, L, l, K, k);
              N[(((long)g * nauxV + nu) * nV + j) * nK + k] += acc;
            }
      }
    }
    /* G_{jk}(R1 - R) index */
    int iRjk = bvk(s, R1[0] - Rv[0], R1[1] - Rv[1], R1[2] - Rv[2]);
    double *O = (double *)malloc(sizeof(double) * (size_t)nU * nK);
    for (int nu = 0; nu < nauxV; ++nu) {
      for (int i = 0; i < nU; ++i)
        for (int k = 0; k < nK; ++k) {
          double m = 0.0, mstar = 0.0, z = 0.0, zstar = 0.0;
          for (int j = 0; j < nV; ++j) {
            /* M = G^vir_{ij}(R) N[G^occ]; M*(-i tau) = G^occ_{ij}(R) N[G^vir] */
            m += gel(s, Ga, iR, U, i, V, j) * N[(((long)0 * nauxV + nu) * nV + j) * nK + k];
            mstar += gel(s, Gb, iR, U, i, V, j) * N[(((long)1 * nauxV + nu) * nV + j) * nK + k];
            /* Z = G^occ_{jk}(R1 - R) X[G^vir]; Z*(-i tau) = G^vir_{jk}(R1 - R) X[G^occ] */
            z += gel(s, Gb, iRjk, V, j, K, k) * X[(((long)0 * nauxV + nu) * nU + i) * nV + j];
            zstar += gel(s, Ga, iRjk, V, j, K, k) * X[(((long)1 * nauxV + nu) * nU + i) * nV + j];
          }
          O[(long)i * nK + k] = m + mstar + z + zstar;
        }
      for (int mu = 0; mu < nauxU; ++mu) {
        double acc = 0.0;
        for (int i = 0; i < nU; ++i)
          for (int k = 0; k < nK; ++k) acc += CU[((long)mu * nU + i) * nK + k] * O[(long)i * nK + k];
        out[(long)mu * ldo + nu] += acc;
      }
    }
    free(O);
    free(N);
  }
  free(X);
}

/*
 * chi0(R, tau) = -spin * sum C O for the requested points.
 *   pts[2*p + 0] = BvK index of R, pts[2*p + 1] = tau index;
 *   pairs: npairs (U, V) pairs, or npairs = 0 for all;
 *   out: [npts][naux][naux], only the requested blocks are written (others untouched).
 */
int oracle_chi0_alg1(int natoms, const int *n_ao, const int *n_aux, const int *kmesh, int nblk,
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
  build_lists(&s);
  const long gstride = (long)s.nR * s.nao * s.nao;
  const int np = npairs > 0 ? npairs : natoms * natoms;
  const long nwork = (long)npts * np;
#pragma omp parallel for schedule(dynamic, 1)
  for (long w = 0; w < nwork; ++w) {
    int p = (int)(w / np), q = (int)(w % np);
    int U = npairs > 0 ? pairs[2 * q] : q / natoms;
    int V = npairs > 0 ? pairs[2 * q + 1] : q % natoms;
    int iR = pts[2 * p], it = pts[2 * p + 1];
    if (it < 0 || it >= ntau || iR < 0 || iR >= s.nR) continue;
    int Rv[3] = {iR / (s.nk2 * s.nk3), (iR / s.nk3) % s.nk2, iR % s.nk3};
    double *blk = (double *)calloc((size_t)n_aux[U] * n_aux[V], sizeof(double));
    pair_block(&s, U, V, Rv, iR, Gv + it * gstride, Go + it * gstride, blk, n_aux[V]);
    double *dst = out + (long)p * s.naux * s.naux;
    for (int mu = 0; mu < n_aux[U]; ++mu)
      for (int nu = 0; nu < n_aux[V]; ++nu)
        dst[(long)(aux_off[U] + mu) * s.naux + aux_off[V] + nu] = -spin * blk[(long)mu * n_aux[V] + nu];
    free(blk);
  }
  free(s.first);
  free(s.order);
  free(ao_off);
  free(aux_off);
  return 0;
}
