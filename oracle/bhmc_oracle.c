/*
 * bhmc_oracle.c -- plain FP64 CPU oracle of the Barnes-Hut octree Monte Carlo
 * method for charged systems (Gan & Xu, Sci. China Math. 2013).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the package smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  It shares no code
 * with the CUDA library.  Build: gcc -O2 -ffp-contract=off -fno-fast-math.
 *
 * The code follows the paper's steps in the paper's order and notation:
 *   Eq. (1.1)          total energy by direct summation
 *   Eq. (3.3)          p-th order particle-cluster approximation
 *                      l_B q_i sum_{||n||<=p} T_n(r_A - r_i) M_A^n
 *   Sec. 3.1           recurrence for the Taylor coefficients T_n
 *   Eq. (3.4)          truncation bound (per-order form, see or_visit)
 *   Sec. 3.2           octree: every cluster keeps N_A, rho_A, its box, level,
 *                      an index array of all its particles, its moments and the
 *                      eight children; traversal with the MAC and N_0
 *   Sec. 3.3           local adjustment: per level, stay -> update moments,
 *                      change -> delete (swap with last, fix tracking) + add
 *                      (append); tracking = per particle, per level, its cluster
 *                      and its position in that cluster's index array
 *   Sec. 2             Metropolis acceptance alpha <= exp(-beta dV)
 * Readings where the paper is silent (all stated in the design notes):
 *   - the root is a fixed dyadic cube; a trial position outside it is rejected;
 *   - octant ties (x == centre) go to the upper child;
 *   - adaptive tree: a cluster is split while it holds more than C charges and
 *     is above level Dmax (the paper's fixed level L_max is the special case of
 *     splitting every non-empty cluster down to Dmax);
 *   - after a move, the topmost cluster on an old path that is internal with at
 *     most C charges is merged into a leaf, and a leaf on a new path holding more
 *     than C charges is split, so the tree is a function of the particle set;
 *   - no depth-Dmax cell may hold more than C charges (a move that would break
 *     this is rejected);
 *   - cluster centre r_A = geometric box centre; MAC in the squared form
 *     rho_A^2 <= theta^2 |r_A - x|^2 with a fixed operation order;
 *   - the moved ion and its image are excluded from the tree while the energy
 *     at the old and the new positions is evaluated on the pre-move tree;
 *   - images are plain point charges in the tree: position R^2 r/|r|^2, charge
 *     alpha q R/|r|, moving with their ion.
 */
#include "bhmc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
   as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with Weyl key
   increments. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* ------------------------------------------------------------------------- */
/* Multi-indices n = (n1, n2, n3), ||n|| <= p, in graded order: k = 0..p; within
   an order n1 runs from k down to 0 and, for each n1, n2 from k - n1 down to 0. */
int or_nterms(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

int or_term_index(int n1, int n2, int n3) {
  int k = n1 + n2 + n3;
  int a = k - n1;
  return k * (k + 1) * (k + 2) / 6 + a * (a + 1) / 2 + (a - n2);
}

/* T_n(R) = (1/n!) D^n f(R), f(r) = 1/|r|, from the recurrence of Sec. 3.1:
     ||n|| r^2 T_n + (2||n|| - 1) sum_i x_i T_{n-e_i} + (||n|| - 1) sum_i T_{n-2e_i} = 0,
   T_0 = 1/r, T_n = 0 when any index is negative. */
int or_taylor(int p, const double R[3], double* T) {
  if (p < 0 || p > OR_PMAX) return OR_EINVAL;
  static __thread double t[OR_PMAX + 1][OR_PMAX + 1][OR_PMAX + 1];
  double r2 = (R[0] * R[0] + R[1] * R[1]) + R[2] * R[2];
  t[0][0][0] = 1.0 / sqrt(r2);
  for (int k = 1; k <= p; ++k) {
    for (int n1 = k; n1 >= 0; --n1) {
      for (int n2 = k - n1; n2 >= 0; --n2) {
        int n3 = k - n1 - n2;
        double s1 = 0.0, s2 = 0.0;
        if (n1 >= 1) s1 += R[0] * t[n1 - 1][n2][n3];
        if (n2 >= 1) s1 += R[1] * t[n1][n2 - 1][n3];
        if (n3 >= 1) s1 += R[2] * t[n1][n2][n3 - 1];
        if (n1 >= 2) s2 += t[n1 - 2][n2][n3];
        if (n2 >= 2) s2 += t[n1][n2 - 2][n3];
        if (n3 >= 2) s2 += t[n1][n2][n3 - 2];
        t[n1][n2][n3] = -((2.0 * k - 1.0) * s1 + (k - 1.0) * s2) / (k * r2);
      }
    }
  }
  for (int k = 0; k <= p; ++k)
    for (int n1 = k; n1 >= 0; --n1)
      for (int n2 = k - n1; n2 >= 0; --n2) {
        int n3 = k - n1 - n2;
        T[or_term_index(n1, n2, n3)] = t[n1][n2][n3];
      }
  return OR_OK;
}

/* q * (d1^n1 d2^n2 d3^n3) for every ||n|| <= p, graded order (the summand of
   M_A^n in Eq. (3.3)). */
static void or_monomials(int p, double q, const double d[3], double* out) {
  double px[OR_PMAX + 1], py[OR_PMAX + 1], pz[OR_PMAX + 1];
  px[0] = py[0] = pz[0] = 1.0;
  for (int k = 1; k <= p; ++k) {
    px[k] = px[k - 1] * d[0];
    py[k] = py[k - 1] * d[1];
    pz[k] = pz[k - 1] * d[2];
  }
  for (int k = 0; k <= p; ++k)
    for (int n1 = k; n1 >= 0; --n1)
      for (int n2 = k - n1; n2 >= 0; --n2) {
        int n3 = k - n1 - n2;
        out[or_term_index(n1, n2, n3)] = q * ((px[n1] * py[n2]) * pz[n3]);
      }
}

double or_direct_energy_raw(int64_t n, const double* q, const double* xyz, double lB) {
  double E = 0.0;
  for (int64_t i = 0; i < n - 1; ++i)
    for (int64_t j = i + 1; j < n; ++j) {
      double dx = xyz[3 * i] - xyz[3 * j];
      double dy = xyz[3 * i + 1] - xyz[3 * j + 1];
      double dz = xyz[3 * i + 2] - xyz[3 * j + 2];
      E += q[i] * q[j] / sqrt((dx * dx + dy * dy) + dz * dz);
    }
  return lB * E;
}

/* ------------------------------------------------------------------------- */
/* The octree of Sec. 3.2. */
typedef struct {
  int depth;      /* level l_A */
  uint64_t key;   /* Morton path: 1 at the root, (parent << 3) | octant below */
  double c[3];    /* middle values of the box (cluster centre r_A) */
  double h;       /* half side: min = c - h, max = c + h, rho_A = sqrt(3) h */
  int child;      /* first of eight contiguous children, -1 for a leaf */
  int alive;
  int64_t n, cap; /* N_A and the index array of all particles in A */
  int64_t* idx;
  double* M;      /* moments M_A^n, graded order */
} or_node;

struct or_sys {
  or_params P;
  int64_t n_mob, n_fix, n_tot;
  int K, L; /* K(p) terms; L = Dmax + 1 levels */
  double theta2;
  int want_bound;
  double* x; /* n_tot x 3 */
  double* q;
  uint64_t* key;   /* depth-Dmax Morton key of every charge */
  int* node_of;    /* tracking: cluster of charge j at level d, -1 below its leaf */
  int64_t* slot_of;/* tracking: position of j in that cluster's index array */
  or_node* nodes;
  int n_nodes, cap_nodes;
  int* free_groups;
  int n_free, cap_free;
  double* scratch; /* 4 K(p) doubles */
};

static int is_pow2(double v) {
  int e;
  double m = frexp(v, &e);
  return v > 0.0 && m == 0.5;
}

int64_t or_n_charges(const or_sys* s) { return s->n_tot; }

void or_get_charges(const or_sys* s, double* q, double* xyz) {
  memcpy(q, s->q, sizeof(double) * s->n_tot);
  memcpy(xyz, s->x, sizeof(double) * 3 * s->n_tot);
}

static int64_t img_index(const or_sys* s, int64_t i) { return s->n_mob + s->n_fix + i; }

/* With fixed_direct, the fixed charges n_mob .. n_mob + n_fix - 1 are not in the tree. */
static int is_fixed(const or_sys* s, int64_t j) { return j >= s->n_mob && j < s->n_mob + s->n_fix; }
static int in_tree(const or_sys* s, int64_t j) { return !(s->P.fixed_direct && is_fixed(s, j)); }

int or_image_of(const or_sys* s, const double r[3], double q, double rim[3], double* qim) {
  double R = s->P.image_R;
  double r2 = (r[0] * r[0] + r[1] * r[1]) + r[2] * r[2];
  if (!(r2 > 0.0)) return OR_EDOMAIN;
  double rn = sqrt(r2);
  double f = (R * R) / r2;
  rim[0] = f * r[0];
  rim[1] = f * r[1];
  rim[2] = f * r[2];
  *qim = ((s->P.image_alpha * q) * R) / rn;
  return OR_OK;
}

static int in_root(const or_sys* s, const double x[3]) {
  for (int a = 0; a < 3; ++a) {
    double lo = s->P.root_lo[a];
    double hi = lo + s->P.root_side;
    if (!(x[a] >= lo) || !(x[a] < hi)) return 0;
  }
  return 1;
}

static int shell_ok(const or_sys* s, const double x[3]) {
  if (!s->P.shell) return 1;
  double r2 = (x[0] * x[0] + x[1] * x[1]) + x[2] * x[2];
  double lo = s->P.shell_rmin * s->P.shell_rmin;
  double hi = s->P.shell_rmax * s->P.shell_rmax;
  return r2 >= lo && r2 <= hi;
}

/* Octant of a point relative to a box centre; ties go to the upper child. */
static int octant(const double c[3], const double x[3]) {
  return (x[0] >= c[0] ? 1 : 0) | (x[1] >= c[1] ? 2 : 0) | (x[2] >= c[2] ? 4 : 0);
}

static void child_centre(const double c[3], double h, int o, double out[3]) {
  double hc = 0.5 * h;
  out[0] = (o & 1) ? c[0] + hc : c[0] - hc;
  out[1] = (o & 2) ? c[1] + hc : c[1] - hc;
  out[2] = (o & 4) ? c[2] + hc : c[2] - hc;
}

uint64_t or_point_key(const or_sys* s, const double x[3]) {
  if (!in_root(s, x)) return 0;
  double h = 0.5 * s->P.root_side;
  double c[3] = {s->P.root_lo[0] + h, s->P.root_lo[1] + h, s->P.root_lo[2] + h};
  uint64_t k = 1;
  for (int d = 1; d <= s->P.Dmax; ++d) {
    int o = octant(c, x);
    double cc[3];
    child_centre(c, h, o, cc);
    memcpy(c, cc, sizeof c);
    h *= 0.5;
    k = (k << 3) | (uint64_t)o;
  }
  return k;
}

static int* track_node(or_sys* s, int64_t j, int d) { return &s->node_of[j * s->L + d]; }
static int64_t* track_slot(or_sys* s, int64_t j, int d) { return &s->slot_of[j * s->L + d]; }

static void idx_push(or_node* A, int64_t j) {
  if (A->n == A->cap) {
    int64_t nc = A->cap ? 2 * A->cap : 8;
    A->idx = (int64_t*)realloc(A->idx, sizeof(int64_t) * nc);
    A->cap = nc;
  }
  A->idx[A->n++] = j;
}

static int alloc_group(or_sys* s) {
  int g;
  if (s->n_free > 0) {
    g = s->free_groups[--s->n_free];
  } else {
    if (s->n_nodes + 8 > s->cap_nodes) {
      int nc = s->cap_nodes * 2 + 64;
      s->nodes = (or_node*)realloc(s->nodes, sizeof(or_node) * nc);
      memset(s->nodes + s->cap_nodes, 0, sizeof(or_node) * (nc - s->cap_nodes));
      s->cap_nodes = nc;
    }
    g = s->n_nodes;
    s->n_nodes += 8;
  }
  for (int o = 0; o < 8; ++o) {
    or_node* A = &s->nodes[g + o];
    if (!A->M) A->M = (double*)malloc(sizeof(double) * s->K);
    A->n = 0;
    A->child = -1;
    A->alive = 1;
  }
  return g;
}

static void push_free(or_sys* s, int g) {
  if (s->n_free == s->cap_free) {
    s->cap_free = s->cap_free * 2 + 16;
    s->free_groups = (int*)realloc(s->free_groups, sizeof(int) * s->cap_free);
  }
  s->free_groups[s->n_free++] = g;
}

/* M_A^n = sum_{j in A} q_j (r_j - r_A)^n, summed in index-array order. */
static void node_moments(or_sys* s, int a) {
  or_node* A = &s->nodes[a];
  double* mono = s->scratch;
  for (int t = 0; t < s->K; ++t) A->M[t] = 0.0;
  for (int64_t k = 0; k < A->n; ++k) {
    int64_t j = A->idx[k];
    double d[3] = {s->x[3 * j] - A->c[0], s->x[3 * j + 1] - A->c[1], s->x[3 * j + 2] - A->c[2]};
    or_monomials(s->P.p, s->q[j], d, mono);
    for (int t = 0; t < s->K; ++t) A->M[t] += mono[t];
  }
}

/* Bisect cluster a in each direction: eight children, the index array
   distributed by octant (Sec. 3.2), children moments computed from scratch. */
static void split_node(or_sys* s, int a) {
  int g = alloc_group(s);
  or_node* A = &s->nodes[a];
  A->child = g;
  for (int o = 0; o < 8; ++o) {
    or_node* Ch = &s->nodes[g + o];
    A = &s->nodes[a];
    Ch->depth = A->depth + 1;
    Ch->key = (A->key << 3) | (uint64_t)o;
    child_centre(A->c, A->h, o, Ch->c);
    Ch->h = 0.5 * A->h;
  }
  A = &s->nodes[a];
  int dc = A->depth + 1;
  for (int64_t k = 0; k < A->n; ++k) {
    int64_t j = A->idx[k];
    int o = octant(A->c, &s->x[3 * j]);
    or_node* Ch = &s->nodes[g + o];
    *track_node(s, j, dc) = g + o;
    *track_slot(s, j, dc) = Ch->n;
    idx_push(Ch, j);
  }
  for (int o = 0; o < 8; ++o) node_moments(s, g + o);
}

/* A cluster above Dmax splits when it holds more than this many charges: C,
   or 0 for the fixed-level tree of Sec. 3.2 (every non-empty cluster is
   bisected down to L_max = Dmax). */
static int split_threshold(const or_params* P) { return P->fixed_depth ? 0 : P->C; }

static void split_rec(or_sys* s, int a) {
  or_node* A = &s->nodes[a];
  if (A->n > split_threshold(&s->P) && A->depth < s->P.Dmax) {
    split_node(s, a);
    int g = s->nodes[a].child;
    for (int o = 0; o < 8; ++o) split_rec(s, g + o);
  }
}

static void free_subtree(or_sys* s, int a) {
  int g = s->nodes[a].child;
  if (g < 0) return;
  for (int o = 0; o < 8; ++o) {
    free_subtree(s, g + o);
    s->nodes[g + o].alive = 0;
    s->nodes[g + o].n = 0;
  }
  s->nodes[a].child = -1;
  push_free(s, g);
}

/* Merge: cluster a becomes a leaf; its own index array already lists all its
   particles, so only the tracking below its level is cleared. */
static void merge_node(or_sys* s, int a) {
  free_subtree(s, a);
  or_node* A = &s->nodes[a];
  for (int64_t k = 0; k < A->n; ++k) {
    int64_t j = A->idx[k];
    for (int d = A->depth + 1; d < s->L; ++d) {
      *track_node(s, j, d) = -1;
      *track_slot(s, j, d) = -1;
    }
  }
}

void or_destroy(or_sys* s) {
  if (!s) return;
  for (int a = 0; a < s->cap_nodes; ++a) {
    free(s->nodes[a].idx);
    free(s->nodes[a].M);
  }
  free(s->nodes);
  free(s->free_groups);
  free(s->x);
  free(s->q);
  free(s->key);
  free(s->node_of);
  free(s->slot_of);
  free(s->scratch);
  free(s);
}

/* Hard core of Eq. (2.1) between mobile ions of common diameter tau: the pair
   potential is infinite for r_ij <= tau, i.e. (dx dx + dy dy) + dz dz <= tau^2. */
static int hard_core_overlap(const or_sys* s, int64_t i, const double b[3]) {
  const double t2 = s->P.hard_core * s->P.hard_core;
  for (int64_t j = 0; j < s->n_mob; ++j) {
    if (j == i) continue;
    const double dx = b[0] - s->x[3 * j], dy = b[1] - s->x[3 * j + 1], dz = b[2] - s->x[3 * j + 2];
    if ((dx * dx + dy * dy) + dz * dz <= t2) return 1;
  }
  return 0;
}

or_sys* or_create(const or_params* P, int64_t n_mob, int64_t n_fix, const double* q,
                  const double* xyz, int* status) {
  *status = OR_EINVAL;
  if (P->p < 0 || P->p > OR_PMAX || P->C < 2 || P->Dmax < 1 || P->Dmax > OR_DMAX || P->N0 < 0)
    return NULL;
  if (!(P->theta >= 0.0 && P->theta < 1.0) || !is_pow2(P->root_side) || n_mob < 0 || n_fix < 0)
    return NULL;
  if (n_mob + n_fix < 1) return NULL;
  or_sys* s = (or_sys*)calloc(1, sizeof(or_sys));
  s->P = *P;
  s->n_mob = n_mob;
  s->n_fix = n_fix;
  s->n_tot = n_mob + n_fix + (P->images ? n_mob : 0);
  s->K = or_nterms(P->p);
  s->L = P->Dmax + 1;
  s->theta2 = P->theta * P->theta;
  s->x = (double*)malloc(sizeof(double) * 3 * s->n_tot);
  s->q = (double*)malloc(sizeof(double) * s->n_tot);
  s->key = (uint64_t*)malloc(sizeof(uint64_t) * s->n_tot);
  s->node_of = (int*)malloc(sizeof(int) * s->n_tot * s->L);
  s->slot_of = (int64_t*)malloc(sizeof(int64_t) * s->n_tot * s->L);
  s->scratch = (double*)malloc(sizeof(double) * 4 * s->K);
  memcpy(s->x, xyz, sizeof(double) * 3 * (n_mob + n_fix));
  memcpy(s->q, q, sizeof(double) * (n_mob + n_fix));
  if (P->images) {
    for (int64_t i = 0; i < n_mob; ++i) {
      int64_t k = img_index(s, i);
      if (or_image_of(s, &s->x[3 * i], s->q[i], &s->x[3 * k], &s->q[k]) != OR_OK) {
        *status = OR_EDOMAIN;
        or_destroy(s);
        return NULL;
      }
    }
  }
  for (int64_t j = 0; j < s->n_tot; ++j) {
    if (!in_root(s, &s->x[3 * j])) {
      *status = OR_EDOMAIN;
      or_destroy(s);
      return NULL;
    }
  }
  for (int64_t i = 0; i < n_mob; ++i) {
    if (!shell_ok(s, &s->x[3 * i])) {
      *status = OR_EOVERLAP;
      or_destroy(s);
      return NULL;
    }
  }
  if (P->hard_core > 0.0) {
    for (int64_t i = 0; i < n_mob; ++i) {
      if (hard_core_overlap(s, i, &s->x[3 * i])) {
        *status = OR_EOVERLAP;
        or_destroy(s);
        return NULL;
      }
    }
  }
  for (int64_t j = 0; j < s->n_tot; ++j) s->key[j] = or_point_key(s, &s->x[3 * j]);
  for (int64_t j = 0; j < s->n_tot * s->L; ++j) {
    s->node_of[j] = -1;
    s->slot_of[j] = -1;
  }
  /* Root cluster (level 0) holds every charge; it is node 0 of an 8-node block
     so that all groups, including the root's, are contiguous blocks of 8. */
  int g = alloc_group(s);
  for (int o = 1; o < 8; ++o) s->nodes[g + o].alive = 0;
  or_node* R = &s->nodes[0];
  R->depth = 0;
  R->key = 1;
  R->h = 0.5 * P->root_side;
  for (int a = 0; a < 3; ++a) R->c[a] = P->root_lo[a] + R->h;
  for (int64_t j = 0; j < s->n_tot; ++j) {
    if (!in_tree(s, j)) continue;
    *track_node(s, j, 0) = 0;
    *track_slot(s, j, 0) = s->nodes[0].n;
    idx_push(&s->nodes[0], j);
  }
  node_moments(s, 0);
  split_rec(s, 0);
  /* capacity rule: no depth-Dmax leaf may hold more than C charges */
  for (int a = 0; a < s->n_nodes; ++a) {
    or_node* A = &s->nodes[a];
    if (A->alive && A->child < 0 && A->n > P->C) {
      *status = OR_ECAPACITY;
      or_destroy(s);
      return NULL;
    }
  }
  *status = OR_OK;
  return s;
}

void or_set_bound(or_sys* s, int on) { s->want_bound = on; }

/* ------------------------------------------------------------------------- */
/* Traversal of Sec. 3.2 for the potential at x of all charges except `excl`.
   Per cluster A, with N'_A = N_A minus the excluded charges inside A:
     N'_A == 0                     -> nothing
     N'_A >= N_0 and MAC holds     -> multipole, Eq. (3.3), with the moments of
                                      A minus the excluded charges' terms
     else A internal, N'_A > N_0   -> examine the eight children
     else                          -> direct sum over A's index array          */
typedef struct {
  const double* x;
  int n_excl;
  const int64_t* excl;
  or_eval* e;
  double* T;
  double* Mp;
  double* mono;
} or_visit_ctx;

static int excluded(const or_visit_ctx* v, int64_t j) {
  for (int k = 0; k < v->n_excl; ++k)
    if (v->excl[k] == j) return 1;
  return 0;
}

static void or_visit(or_sys* s, int a, or_visit_ctx* v) {
  or_node* A = &s->nodes[a];
  int in_a = 0;
  for (int k = 0; k < v->n_excl; ++k)
    if (s->node_of[v->excl[k] * s->L + A->depth] == a) in_a++;
  int64_t Np = A->n - in_a;
  v->e->visited++;
  if (Np == 0) return;
  const double* x = v->x;
  double dx = A->c[0] - x[0];
  double dy = A->c[1] - x[1];
  double dz = A->c[2] - x[2];
  double d2 = (dx * dx + dy * dy) + dz * dz;
  double rho2 = 3.0 * A->h * A->h;
  double rhs = s->theta2 * d2;
  if (fabs(rhs - rho2) <= 0x1p-17 * rho2) v->e->mac_near++;
  if (Np >= s->P.N0 && rho2 <= rhs) {
    /* multipole: M'_A = M_A - sum over excluded charges in A of q (r - r_A)^n */
    int K = s->K;
    for (int t = 0; t < K; ++t) v->Mp[t] = A->M[t];
    for (int k = 0; k < v->n_excl; ++k) {
      int64_t j = v->excl[k];
      if (s->node_of[j * s->L + A->depth] != a) continue;
      double d[3] = {s->x[3 * j] - A->c[0], s->x[3 * j + 1] - A->c[1], s->x[3 * j + 2] - A->c[2]};
      or_monomials(s->P.p, s->q[j], d, v->mono);
      for (int t = 0; t < K; ++t) v->Mp[t] -= v->mono[t];
    }
    double R[3] = {dx, dy, dz}; /* r_A - x */
    or_taylor(s->P.p, R, v->T);
    double sum = 0.0, asum = 0.0;
    for (int t = 0; t < K; ++t) {
      sum += v->T[t] * v->Mp[t];
      asum += fabs(v->T[t] * v->Mp[t]);
    }
    v->e->phi += sum;
    v->e->abs_sum += asum;
    v->e->accepted++;
    if (s->want_bound) {
      /* Eq. (3.4), per order: for |r_j - r_A| <= rho_A the remainder of the
         Taylor series of 1/|r_j - x| beyond order p is at most
         (1/R) gamma^{p+1} / (1 - gamma), gamma = rho_A / R. */
      double Rn = sqrt(d2);
      double gam = sqrt(rho2) / Rn;
      double qabs = 0.0;
      for (int64_t k = 0; k < A->n; ++k)
        if (!excluded(v, A->idx[k])) qabs += fabs(s->q[A->idx[k]]);
      v->e->bound += qabs * pow(gam, s->P.p + 1) / (Rn * (1.0 - gam));
    }
    return;
  }
  if (A->child >= 0 && Np > s->P.N0) {
    int g = A->child;
    for (int o = 0; o < 8; ++o) or_visit(s, g + o, v);
    return;
  }
  for (int64_t k = 0; k < A->n; ++k) {
    int64_t j = A->idx[k];
    if (excluded(v, j)) continue;
    double ex = s->x[3 * j] - x[0];
    double ey = s->x[3 * j + 1] - x[1];
    double ez = s->x[3 * j + 2] - x[2];
    double r = sqrt((ex * ex + ey * ey) + ez * ez);
    v->e->phi += s->q[j] / r;
    v->e->abs_sum += fabs(s->q[j]) / r;
    v->e->pairs++;
  }
}

int or_phi(or_sys* s, const double x[3], int n_excl, const int64_t* excl, or_eval* out) {
  memset(out, 0, sizeof(*out));
  or_visit_ctx v;
  double T[286], Mp[286], mono[286];
  v.x = x;
  v.n_excl = n_excl;
  v.excl = excl;
  v.e = out;
  v.T = T;
  v.Mp = Mp;
  v.mono = mono;
  or_visit(s, 0, &v);
  if (s->P.fixed_direct) {
    /* the fixed charges outside the tree: exact terms q_f / |r_f - x| */
    for (int64_t j = s->n_mob; j < s->n_mob + s->n_fix; ++j) {
      if (excluded(&v, j)) continue;
      double ex = s->x[3 * j] - x[0];
      double ey = s->x[3 * j + 1] - x[1];
      double ez = s->x[3 * j + 2] - x[2];
      double r = sqrt((ex * ex + ey * ey) + ez * ez);
      out->phi += s->q[j] / r;
      out->abs_sum += fabs(s->q[j]) / r;
    }
  }
  return OR_OK;
}

double or_phi_direct(const or_sys* s, const double x[3], int n_excl, const int64_t* excl) {
  double phi = 0.0;
  for (int64_t j = 0; j < s->n_tot; ++j) {
    int skip = 0;
    for (int k = 0; k < n_excl; ++k)
      if (excl[k] == j) skip = 1;
    if (skip) continue;
    double ex = s->x[3 * j] - x[0];
    double ey = s->x[3 * j + 1] - x[1];
    double ez = s->x[3 * j + 2] - x[2];
    phi += s->q[j] / sqrt((ex * ex + ey * ey) + ez * ez);
  }
  return phi;
}

/* ------------------------------------------------------------------------- */
/* Energy difference of a single-particle trial move (Sec. 1: V_i evaluated
   before and after the displacement; Sec. 2 step 2). */
typedef struct {
  double a[3], b[3], ai[3], bi[3];
  double q, qa_img, qb_img;
  int64_t excl[2];
  int n_excl;
} or_move;

static int prepare_move(const or_sys* s, int64_t i, const double b[3], or_move* m) {
  if (i < 0 || i >= s->n_mob) return OR_EINVAL;
  for (int a = 0; a < 3; ++a) {
    m->a[a] = s->x[3 * i + a];
    m->b[a] = b[a];
  }
  m->q = s->q[i];
  m->excl[0] = i;
  m->n_excl = 1;
  if (!in_root(s, b)) return OR_EDOMAIN;
  if (!shell_ok(s, b)) return OR_EOVERLAP;
  if (s->P.images) {
    int64_t k = img_index(s, i);
    for (int a = 0; a < 3; ++a) m->ai[a] = s->x[3 * k + a];
    m->qa_img = s->q[k];
    if (or_image_of(s, b, m->q, m->bi, &m->qb_img) != OR_OK) return OR_EDOMAIN;
    if (!in_root(s, m->bi)) return OR_EDOMAIN;
    m->excl[1] = k;
    m->n_excl = 2;
  }
  if (s->P.hard_core > 0.0 && hard_core_overlap(s, i, b)) return OR_EOVERLAP;
  return OR_OK;
}

static double dist(const double u[3], const double v[3]) {
  double dx = u[0] - v[0], dy = u[1] - v[1], dz = u[2] - v[2];
  return sqrt((dx * dx + dy * dy) + dz * dz);
}

int or_delta_energy(or_sys* s, int64_t i, const double b[3], or_dE* out) {
  memset(out, 0, sizeof(*out));
  or_move m;
  int st = prepare_move(s, i, b, &m);
  out->status = st;
  if (st != OR_OK) return st;
  or_eval ea, eb;
  or_phi(s, m.a, m.n_excl, m.excl, &ea);
  or_phi(s, m.b, m.n_excl, m.excl, &eb);
  double dE = m.q * (eb.phi - ea.phi);
  double A = fabs(m.q) * (ea.abs_sum + eb.abs_sum);
  double B = fabs(m.q) * (ea.bound + eb.bound);
  out->visited = ea.visited + eb.visited;
  out->accepted = ea.accepted + eb.accepted;
  out->pairs = ea.pairs + eb.pairs;
  if (s->P.images) {
    or_eval eai, ebi;
    or_phi(s, m.ai, m.n_excl, m.excl, &eai);
    or_phi(s, m.bi, m.n_excl, m.excl, &ebi);
    dE += m.qb_img * ebi.phi - m.qa_img * eai.phi;
    double pb = m.q * m.qb_img / dist(m.b, m.bi);
    double pa = m.q * m.qa_img / dist(m.a, m.ai);
    dE += pb - pa;
    A += fabs(m.qa_img) * eai.abs_sum + fabs(m.qb_img) * ebi.abs_sum + fabs(pb) + fabs(pa);
    B += fabs(m.qa_img) * eai.bound + fabs(m.qb_img) * ebi.bound;
    out->visited += eai.visited + ebi.visited;
    out->accepted += eai.accepted + ebi.accepted;
    out->pairs += eai.pairs + ebi.pairs;
  }
  out->dE = s->P.lB * dE;
  out->abs_sum = s->P.lB * A;
  out->bound = s->P.lB * B;
  return OR_OK;
}

int or_delta_energy_direct(const or_sys* s, int64_t i, const double b[3], double* dE) {
  or_move m;
  int st = prepare_move(s, i, b, &m);
  if (st != OR_OK) return st;
  double e = m.q * (or_phi_direct(s, m.b, m.n_excl, m.excl) - or_phi_direct(s, m.a, m.n_excl, m.excl));
  if (s->P.images) {
    e += m.qb_img * or_phi_direct(s, m.bi, m.n_excl, m.excl) -
         m.qa_img * or_phi_direct(s, m.ai, m.n_excl, m.excl);
    e += m.q * m.qb_img / dist(m.b, m.bi) - m.q * m.qa_img / dist(m.a, m.ai);
  }
  *dE = s->P.lB * e;
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Local adjustment (Sec. 3.3) of one charge j moving from its position to b
   with charge qb.  Level by level from the root: if the cluster at this level
   is unchanged, its moments are updated; otherwise j is deleted from the old
   cluster (its slot refilled by the last index, whose tracking is fixed) and
   appended to the new one. */
static void move_charge(or_sys* s, int64_t j, const double b[3], double qb) {
  double a[3] = {s->x[3 * j], s->x[3 * j + 1], s->x[3 * j + 2]};
  double qa = s->q[j];
  double* ma = s->scratch;
  double* mb = s->scratch + s->K;
  int K = s->K;
  int A2 = 0; /* new cluster at the current level; -1 below the new leaf */
  for (int d = 0; d < s->L; ++d) {
    int A1 = *track_node(s, j, d);
    if (A1 < 0 && A2 < 0) break;
    if (A1 >= 0 && A1 == A2) {
      or_node* A = &s->nodes[A1];
      double da[3] = {a[0] - A->c[0], a[1] - A->c[1], a[2] - A->c[2]};
      double db[3] = {b[0] - A->c[0], b[1] - A->c[1], b[2] - A->c[2]};
      or_monomials(s->P.p, qa, da, ma);
      or_monomials(s->P.p, qb, db, mb);
      for (int t = 0; t < K; ++t) A->M[t] += mb[t] - ma[t];
    } else {
      if (A1 >= 0) { /* delete from A1 */
        or_node* A = &s->nodes[A1];
        int64_t pos = *track_slot(s, j, d);
        int64_t last = A->idx[A->n - 1];
        A->idx[pos] = last;
        *track_slot(s, last, d) = pos;
        A->n--;
        double da[3] = {a[0] - A->c[0], a[1] - A->c[1], a[2] - A->c[2]};
        or_monomials(s->P.p, qa, da, ma);
        for (int t = 0; t < K; ++t) A->M[t] -= ma[t];
        *track_node(s, j, d) = -1;
        *track_slot(s, j, d) = -1;
      }
      if (A2 >= 0) { /* add to A2 */
        or_node* A = &s->nodes[A2];
        *track_node(s, j, d) = A2;
        *track_slot(s, j, d) = A->n;
        idx_push(A, j);
        A = &s->nodes[A2];
        double db[3] = {b[0] - A->c[0], b[1] - A->c[1], b[2] - A->c[2]};
        or_monomials(s->P.p, qb, db, mb);
        for (int t = 0; t < K; ++t) A->M[t] += mb[t];
      }
    }
    if (A2 >= 0) {
      or_node* A = &s->nodes[A2];
      A2 = (A->child >= 0) ? A->child + octant(A->c, b) : -1;
    }
  }
  for (int a3 = 0; a3 < 3; ++a3) s->x[3 * j + a3] = b[a3];
  s->q[j] = qb;
  s->key[j] = or_point_key(s, b);
}

int or_capacity_violation(or_sys* s, int64_t i, const double b[3]) {
  or_move m;
  if (prepare_move(s, i, b, &m) != OR_OK) return 0;
  const double* pts[2] = {m.b, m.bi};
  int np = s->P.images ? 2 : 1;
  for (int t = 0; t < np; ++t) {
    uint64_t kb = or_point_key(s, pts[t]);
    /* the cell lies inside the current leaf that contains the point */
    int a = 0;
    while (s->nodes[a].child >= 0) a = s->nodes[a].child + octant(s->nodes[a].c, pts[t]);
    int64_t cnt = 0;
    or_node* A = &s->nodes[a];
    for (int64_t k = 0; k < A->n; ++k) {
      int64_t j = A->idx[k];
      if (j == m.excl[0] || (m.n_excl > 1 && j == m.excl[1])) continue;
      if (s->key[j] == kb) cnt++;
    }
    for (int u = 0; u < np; ++u)
      if (or_point_key(s, pts[u]) == kb) cnt++;
    if (cnt > s->P.C) return 1;
  }
  return 0;
}

int or_commit_move(or_sys* s, int64_t i, const double b[3]) {
  or_move m;
  int st = prepare_move(s, i, b, &m);
  if (st != OR_OK) return st;
  if (or_capacity_violation(s, i, b)) return OR_ECAPACITY;
  /* old paths, for the merge test */
  int old_path[2][OR_DMAX + 1];
  for (int t = 0; t < m.n_excl; ++t)
    for (int d = 0; d < s->L; ++d) old_path[t][d] = *track_node(s, m.excl[t], d);
  move_charge(s, i, m.b, m.q);
  if (s->P.images) move_charge(s, m.excl[1], m.bi, m.qb_img);
  /* merge the topmost internal cluster on an old path holding no more charges than the split threshold */
  for (int t = 0; t < m.n_excl; ++t) {
    for (int d = 0; d < s->L; ++d) {
      int a = old_path[t][d];
      if (a < 0) break;
      or_node* A = &s->nodes[a];
      if (!A->alive) break;
      if (A->child >= 0 && A->n <= split_threshold(&s->P)) {
        merge_node(s, a);
        break;
      }
    }
  }
  /* split the new leaves while they hold more charges than the split threshold */
  for (int t = 0; t < m.n_excl; ++t) {
    int64_t j = m.excl[t];
    int leaf = -1;
    for (int d = 0; d < s->L; ++d) {
      int a = *track_node(s, j, d);
      if (a < 0) break;
      leaf = a;
    }
    split_rec(s, leaf);
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Metropolis chain (Sec. 2): choose ion i and a uniform displacement in
   [-step/2, step/2)^3 from Philox block (m, replica, 0); alpha from block
   (m, replica, 1); accept iff alpha <= exp(-beta dE). */
int or_mc_run(or_sys* s, uint64_t seed, uint32_t replica, uint64_t m0, int64_t n_moves,
              double step, or_record* recs, int64_t* n_accepted) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  int64_t acc = 0;
  if (n_moves > 0 && s->n_mob < 1) return OR_EINVAL; /* no mobile ion to move */
  for (int64_t t = 0; t < n_moves; ++t) {
    uint64_t mm = m0 + (uint64_t)t;
    uint32_t ctr[4] = {(uint32_t)mm, (uint32_t)(mm >> 32), replica, 0u};
    uint32_t u[4], v[4];
    or_philox4x32_10(ctr, key, u);
    ctr[3] = 1u;
    or_philox4x32_10(ctr, key, v);
    int64_t i = (int64_t)(((uint64_t)u[0] * (uint64_t)s->n_mob) >> 32);
    double b[3];
    for (int a = 0; a < 3; ++a) {
      double delta = (((double)u[a + 1] * 0x1p-32 + 0x1p-33) - 0.5) * step;
      b[a] = s->x[3 * i + a] + delta;
    }
    double alpha = ((double)v[0] + 0.5) * 0x1p-32;
    or_record r;
    memset(&r, 0, sizeof r);
    r.i = i;
    memcpy(r.r_new, b, sizeof b);
    r.log_alpha = log(alpha);
    or_dE e;
    int st = or_delta_energy(s, i, b, &e);
    if (st == OR_EDOMAIN) {
      r.outcome = OR_REJECT_DOMAIN;
    } else if (st == OR_EOVERLAP) {
      r.outcome = OR_REJECT_OVERLAP;
    } else {
      r.dE = e.dE;
      r.abs_sum = e.abs_sum;
      int accept = alpha <= exp(-s->P.beta * e.dE);
      r.flagged = fabs(s->P.beta * e.dE + r.log_alpha) < 1e-6;
      if (!accept) {
        r.outcome = OR_REJECT_ENERGY;
      } else if (or_capacity_violation(s, i, b)) {
        r.outcome = OR_REJECT_CAPACITY;
      } else {
        or_commit_move(s, i, b);
        r.outcome = OR_ACCEPT;
        acc++;
      }
    }
    if (recs) recs[t] = r;
  }
  if (n_accepted) *n_accepted = acc;
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
double or_energy_direct(const or_sys* s) {
  return or_direct_energy_raw(s->n_tot, s->q, s->x, s->P.lB);
}

/* Potential at charge j from all other charges: the treecode for a charge in
   the tree, the exact sum for a fixed charge outside it (fixed_direct). */
static double target_phi(or_sys* s, int64_t j) {
  double x[3] = {s->x[3 * j], s->x[3 * j + 1], s->x[3 * j + 2]};
  if (!in_tree(s, j)) return or_phi_direct(s, x, 1, &j);
  or_eval e;
  or_phi(s, x, 1, &j, &e);
  return e.phi;
}

/* E_tree = (1/2) l_B sum_i q_i phi_tree(r_i), each charge excluded from its own sum. */
double or_energy_tree(or_sys* s) {
  double E = 0.0;
  for (int64_t j = 0; j < s->n_tot; ++j) E += s->q[j] * target_phi(s, j);
  return 0.5 * s->P.lB * E;
}

int or_potentials(or_sys* s, double* v_tree, double* v_direct) {
  for (int64_t j = 0; j < s->n_tot; ++j) {
    double x[3] = {s->x[3 * j], s->x[3 * j + 1], s->x[3 * j + 2]};
    if (v_tree) v_tree[j] = s->P.lB * s->q[j] * target_phi(s, j);
    if (v_direct) v_direct[j] = s->P.lB * s->q[j] * or_phi_direct(s, x, 1, &j);
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
static int cmp_i64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return (x > y) - (x < y);
}

typedef struct {
  int64_t* rows;
  int64_t max_rows, n_rows;
  int64_t* members;
  int64_t max_members, n_members;
  int overflow;
} or_export_ctx;

static void export_rec(const or_sys* s, int a, or_export_ctx* x) {
  const or_node* A = &s->nodes[a];
  if (x->n_rows >= x->max_rows) {
    x->overflow = 1;
    return;
  }
  int64_t* r = &x->rows[4 * x->n_rows++];
  r[0] = A->depth;
  r[1] = (int64_t)A->key;
  r[2] = A->child < 0;
  r[3] = A->n;
  if (A->child < 0) {
    if (x->n_members + A->n > x->max_members) {
      x->overflow = 1;
      return;
    }
    int64_t* dst = &x->members[x->n_members];
    memcpy(dst, A->idx, sizeof(int64_t) * A->n);
    qsort(dst, A->n, sizeof(int64_t), cmp_i64);
    x->n_members += A->n;
  } else {
    for (int o = 0; o < 8; ++o) export_rec(s, A->child + o, x);
  }
}

int64_t or_export_tree(const or_sys* s, int64_t* rows, int64_t max_rows, int64_t* members,
                       int64_t max_members) {
  or_export_ctx x = {rows, max_rows, 0, members, max_members, 0, 0};
  export_rec(s, 0, &x);
  return x.overflow ? -1 : x.n_rows;
}

static int check_rec(const or_sys* s, int a, int64_t* seen) {
  const or_node* A = &s->nodes[a];
  if (!A->alive) return 1;
  for (int64_t k = 0; k < A->n; ++k) {
    int64_t j = A->idx[k];
    if (s->node_of[j * s->L + A->depth] != a) return 2;
    if (s->slot_of[j * s->L + A->depth] != k) return 3;
    for (int ax = 0; ax < 3; ++ax) {
      double v = s->x[3 * j + ax];
      if (!(v >= A->c[ax] - A->h) || !(v < A->c[ax] + A->h)) return 4;
    }
    if ((s->key[j] >> (3 * (s->P.Dmax - A->depth))) != A->key) return 5;
  }
  if (A->child >= 0) {
    if (!(A->n > split_threshold(&s->P) && A->depth < s->P.Dmax)) return 6;
    int64_t sum = 0;
    for (int o = 0; o < 8; ++o) {
      const or_node* Ch = &s->nodes[A->child + o];
      if (Ch->depth != A->depth + 1 || Ch->key != ((A->key << 3) | (uint64_t)o)) return 7;
      sum += Ch->n;
      int rc = check_rec(s, A->child + o, seen);
      if (rc) return rc;
    }
    if (sum != A->n) return 8;
  } else {
    if (!(A->n <= (A->depth < s->P.Dmax ? split_threshold(&s->P) : s->P.C))) return 9; /* capacity rule at Dmax */
    for (int64_t k = 0; k < A->n; ++k) {
      int64_t j = A->idx[k];
      if (seen[j]) return 10;
      seen[j] = 1;
      for (int d = A->depth + 1; d < s->L; ++d)
        if (s->node_of[j * s->L + d] != -1) return 11;
    }
  }
  return 0;
}

int or_check(const or_sys* s) {
  int64_t* seen = (int64_t*)calloc(s->n_tot, sizeof(int64_t));
  int rc = check_rec(s, 0, seen);
  if (!rc)
    for (int64_t j = 0; j < s->n_tot; ++j)
      if (seen[j] != in_tree(s, j)) {
        rc = 12;
        break;
      }
  free(seen);
  return rc;
}

int or_node_moments(const or_sys* s, int depth, uint64_t key, double* M) {
  for (int a = 0; a < s->n_nodes; ++a) {
    const or_node* A = &s->nodes[a];
    if (A->alive && A->depth == depth && A->key == key) {
      memcpy(M, A->M, sizeof(double) * s->K);
      return OR_OK;
    }
  }
  return OR_EINVAL;
}

/* ------------------------------------------------------------------------- */
/* Exact gradient of E_tree = (1/2) l_B sum_i q_i phi_i with every MAC decision
   held fixed.  phi_i = sum over accepted clusters A of sum_n T_n(r_A - r_i) M_A^n
   + sum over direct partners j of q_j/|r_j - r_i|.
     target side:  d/dr_i of phi_i, with d/dx T_n(r_A - x) = -(n_k + 1) T_{n+e_k}
     source side:  a direct pair (i, j) gives q_i q_j d/dr_j 1/|r_j - r_i| and
                   q_i/|r_j - r_i| to dE/dq_j; an accepted cluster A gives the
                   adjoint lambda_A^n += q_i T_n(r_A - r_i), returned to every
                   member k of A as sum_n lambda_A^n (r_k - r_A)^n (dE/dq_k) and
                   q_k sum_n lambda_A^n d/dr_k (r_k - r_A)^n (dE/dr_k).
   dEdr is n x 3, dEdq is n. */
typedef struct {
  double* lam;   /* n_nodes x K cluster adjoints */
  double* src;   /* n x 3 source-side gradients (direct pairs) */
  double* dq;    /* n source-side charge derivatives (direct pairs) */
  double* T1;    /* Taylor coefficients up to order p + 1 */
  int64_t target;
  double x[3];
  double phi;    /* phi_i */
  double tg[3];  /* grad phi_i (target side) */
  int absm;      /* 1: accumulate |term| instead of term (conditioning sums) */
} or_adj;

/* A term as accumulated: itself, or its magnitude in the conditioning mode. */
static double adj_term(const or_adj* v, double t) { return v->absm ? fabs(t) : t; }

/* One exact pair (target v->target, source j): potential, target gradient and
   the source side's position and charge derivatives. */
static void or_adj_pair(or_sys* s, int64_t j, or_adj* v) {
  int64_t i = v->target;
  double ex = s->x[3 * j] - v->x[0], ey = s->x[3 * j + 1] - v->x[1], ez = s->x[3 * j + 2] - v->x[2];
  double r2 = (ex * ex + ey * ey) + ez * ez;
  double r = sqrt(r2), r3 = r2 * r;
  v->phi += adj_term(v, s->q[j] / r);
  /* target: d/dx q_j/|r_j - x| = q_j (r_j - x)/r^3 */
  v->tg[0] += adj_term(v, s->q[j] * ex / r3);
  v->tg[1] += adj_term(v, s->q[j] * ey / r3);
  v->tg[2] += adj_term(v, s->q[j] * ez / r3);
  /* source: q_i q_j d/dr_j 1/|r_j - r_i| = -q_i q_j (r_j - r_i)/r^3 */
  v->src[3 * j + 0] += adj_term(v, -(s->q[i] * s->q[j] * ex / r3));
  v->src[3 * j + 1] += adj_term(v, -(s->q[i] * s->q[j] * ey / r3));
  v->src[3 * j + 2] += adj_term(v, -(s->q[i] * s->q[j] * ez / r3));
  v->dq[j] += adj_term(v, s->q[i] / r);
}

static void or_adj_visit(or_sys* s, int a, or_adj* v) {
  or_node* A = &s->nodes[a];
  int64_t i = v->target;
  int self = s->node_of[i * s->L + A->depth] == a;
  int64_t Np = A->n - self;
  if (Np == 0) return;
  double dx = A->c[0] - v->x[0], dy = A->c[1] - v->x[1], dz = A->c[2] - v->x[2];
  double d2 = (dx * dx + dy * dy) + dz * dz;
  double rho2 = 3.0 * A->h * A->h;
  int p = s->P.p, K = s->K;
  if (Np >= s->P.N0 && rho2 <= s->theta2 * d2) {
    /* an accepted cluster never contains its target (theta < 1), so M' = M */
    double R[3] = {dx, dy, dz};
    or_taylor(p + 1, R, v->T1);
    for (int k = 0; k <= p; ++k)
      for (int n1 = k; n1 >= 0; --n1)
        for (int n2 = k - n1; n2 >= 0; --n2) {
          int n3 = k - n1 - n2;
          int t = or_term_index(n1, n2, n3);
          double Tn = v->T1[t], Mn = A->M[t];
          v->phi += adj_term(v, Tn * Mn);
          v->tg[0] += adj_term(v, -((n1 + 1) * v->T1[or_term_index(n1 + 1, n2, n3)] * Mn));
          v->tg[1] += adj_term(v, -((n2 + 1) * v->T1[or_term_index(n1, n2 + 1, n3)] * Mn));
          v->tg[2] += adj_term(v, -((n3 + 1) * v->T1[or_term_index(n1, n2, n3 + 1)] * Mn));
          v->lam[(int64_t)a * K + t] += adj_term(v, s->q[i] * Tn);
        }
    return;
  }
  if (A->child >= 0 && Np > s->P.N0) {
    for (int o = 0; o < 8; ++o) or_adj_visit(s, A->child + o, v);
    return;
  }
  for (int64_t k = 0; k < A->n; ++k) {
    int64_t j = A->idx[k];
    if (j == i) continue;
    or_adj_pair(s, j, v);
  }
}

static int or_forces_impl(or_sys* s, double* dEdr, double* dEdq, int absm) {
  int K = s->K, p = s->P.p;
  if (p + 1 > OR_PMAX) return OR_EINVAL; /* orders up to p + 1 enter the target gradient */
  or_adj v;
  v.absm = absm;
  v.lam = (double*)calloc((size_t)s->n_nodes * K, sizeof(double));
  v.src = (double*)calloc((size_t)s->n_tot * 3, sizeof(double));
  v.dq = (double*)calloc((size_t)s->n_tot, sizeof(double));
  v.T1 = (double*)malloc(sizeof(double) * or_nterms(OR_PMAX));
  double* phi = (double*)calloc((size_t)s->n_tot, sizeof(double));
  double* tgt = (double*)calloc((size_t)s->n_tot * 3, sizeof(double));
  for (int64_t i = 0; i < s->n_tot; ++i) {
    v.target = i;
    for (int c = 0; c < 3; ++c) {
      v.x[c] = s->x[3 * i + c];
      v.tg[c] = 0.0;
    }
    v.phi = 0.0;
    if (in_tree(s, i)) {
      or_adj_visit(s, 0, &v);
      /* fixed_direct: the fixed charges outside the tree, exact pairs */
      if (s->P.fixed_direct)
        for (int64_t j = s->n_mob; j < s->n_mob + s->n_fix; ++j) or_adj_pair(s, j, &v);
    } else {
      /* a fixed charge outside the tree: exact pairs with every other charge */
      for (int64_t j = 0; j < s->n_tot; ++j)
        if (j != i) or_adj_pair(s, j, &v);
    }
    phi[i] = v.phi;
    for (int c = 0; c < 3; ++c) tgt[3 * i + c] = adj_term(&v, s->q[i]) * v.tg[c];
  }
  /* cluster adjoints back to their members: every cluster containing charge k */
  for (int64_t k = 0; k < s->n_tot; ++k) {
    double gq = 0.0, gr[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < s->L; ++d) {
      int a = s->node_of[k * s->L + d];
      if (a < 0) break;
      or_node* A = &s->nodes[a];
      double r[3] = {s->x[3 * k] - A->c[0], s->x[3 * k + 1] - A->c[1], s->x[3 * k + 2] - A->c[2]};
      double px[OR_PMAX + 1], py[OR_PMAX + 1], pz[OR_PMAX + 1];
      px[0] = py[0] = pz[0] = 1.0;
      for (int e = 1; e <= p; ++e) {
        px[e] = px[e - 1] * r[0];
        py[e] = py[e - 1] * r[1];
        pz[e] = pz[e - 1] * r[2];
      }
      for (int kk = 0; kk <= p; ++kk)
        for (int n1 = kk; n1 >= 0; --n1)
          for (int n2 = kk - n1; n2 >= 0; --n2) {
            int n3 = kk - n1 - n2;
            double l = v.lam[(int64_t)a * K + or_term_index(n1, n2, n3)];
            gq += adj_term(&v, l * ((px[n1] * py[n2]) * pz[n3]));
            if (n1) gr[0] += adj_term(&v, l * n1 * ((px[n1 - 1] * py[n2]) * pz[n3]));
            if (n2) gr[1] += adj_term(&v, l * n2 * ((px[n1] * py[n2 - 1]) * pz[n3]));
            if (n3) gr[2] += adj_term(&v, l * n3 * ((px[n1] * py[n2]) * pz[n3 - 1]));
          }
    }
    double h = 0.5 * s->P.lB;
    if (dEdq) dEdq[k] = h * (phi[k] + v.dq[k] + gq);
    if (dEdr)
      for (int c = 0; c < 3; ++c)
        dEdr[3 * k + c] = h * (tgt[3 * k + c] + v.src[3 * k + c] + adj_term(&v, s->q[k]) * gr[c]);
  }
  free(v.lam);
  free(v.src);
  free(v.dq);
  free(v.T1);
  free(phi);
  free(tgt);
  return OR_OK;
}

int or_forces(or_sys* s, double* dEdr, double* dEdq) { return or_forces_impl(s, dEdr, dEdq, 0); }

int or_forces_abs(or_sys* s, double* Ar, double* Aq) { return or_forces_impl(s, Ar, Aq, 1); }

/* ------------------------------------------------------------------------- */
/* Potential and its gradient at x (same traversal and exclusions as or_phi). */
typedef struct {
  const double* x;
  int n_excl;
  const int64_t* excl;
  double phi, g[3];
  double* T1;
  double* Mp;
  double* mono;
} or_grad_ctx;

static int excl_has(const or_grad_ctx* v, int64_t j) {
  for (int k = 0; k < v->n_excl; ++k)
    if (v->excl[k] == j) return 1;
  return 0;
}

static void or_grad_visit(or_sys* s, int a, or_grad_ctx* v) {
  or_node* A = &s->nodes[a];
  int in_a = 0;
  for (int k = 0; k < v->n_excl; ++k)
    if (s->node_of[v->excl[k] * s->L + A->depth] == a) in_a++;
  int64_t Np = A->n - in_a;
  if (Np == 0) return;
  const double* x = v->x;
  double dx = A->c[0] - x[0], dy = A->c[1] - x[1], dz = A->c[2] - x[2];
  double d2 = (dx * dx + dy * dy) + dz * dz;
  double rho2 = 3.0 * A->h * A->h;
  int p = s->P.p, K = s->K;
  if (Np >= s->P.N0 && rho2 <= s->theta2 * d2) {
    for (int t = 0; t < K; ++t) v->Mp[t] = A->M[t];
    for (int k = 0; k < v->n_excl; ++k) {
      int64_t j = v->excl[k];
      if (s->node_of[j * s->L + A->depth] != a) continue;
      double d[3] = {s->x[3 * j] - A->c[0], s->x[3 * j + 1] - A->c[1], s->x[3 * j + 2] - A->c[2]};
      or_monomials(p, s->q[j], d, v->mono);
      for (int t = 0; t < K; ++t) v->Mp[t] -= v->mono[t];
    }
    double R[3] = {dx, dy, dz};
    or_taylor(p + 1, R, v->T1);
    for (int k = 0; k <= p; ++k)
      for (int n1 = k; n1 >= 0; --n1)
        for (int n2 = k - n1; n2 >= 0; --n2) {
          int n3 = k - n1 - n2;
          double M = v->Mp[or_term_index(n1, n2, n3)];
          v->phi += v->T1[or_term_index(n1, n2, n3)] * M;
          v->g[0] -= (n1 + 1) * v->T1[or_term_index(n1 + 1, n2, n3)] * M;
          v->g[1] -= (n2 + 1) * v->T1[or_term_index(n1, n2 + 1, n3)] * M;
          v->g[2] -= (n3 + 1) * v->T1[or_term_index(n1, n2, n3 + 1)] * M;
        }
    return;
  }
  if (A->child >= 0 && Np > s->P.N0) {
    for (int o = 0; o < 8; ++o) or_grad_visit(s, A->child + o, v);
    return;
  }
  for (int64_t k = 0; k < A->n; ++k) {
    int64_t j = A->idx[k];
    if (excl_has(v, j)) continue;
    double ex = s->x[3 * j] - x[0], ey = s->x[3 * j + 1] - x[1], ez = s->x[3 * j + 2] - x[2];
    double r2 = (ex * ex + ey * ey) + ez * ez, r = sqrt(r2), r3 = r2 * r;
    v->phi += s->q[j] / r;
    v->g[0] += s->q[j] * ex / r3;
    v->g[1] += s->q[j] * ey / r3;
    v->g[2] += s->q[j] * ez / r3;
  }
}

int or_phi_grad(or_sys* s, const double x[3], int n_excl, const int64_t* excl, double* phi, double g[3]) {
  if (s->P.p + 1 > OR_PMAX) return OR_EINVAL;
  double T1[286], Mp[286], mono[286];
  or_grad_ctx v = {x, n_excl, excl, 0.0, {0.0, 0.0, 0.0}, T1, Mp, mono};
  or_grad_visit(s, 0, &v);
  if (s->P.fixed_direct) {
    /* the fixed charges outside the tree: exact terms and their gradients */
    for (int64_t j = s->n_mob; j < s->n_mob + s->n_fix; ++j) {
      if (excl_has(&v, j)) continue;
      double ex = s->x[3 * j] - x[0], ey = s->x[3 * j + 1] - x[1], ez = s->x[3 * j + 2] - x[2];
      double r2 = (ex * ex + ey * ey) + ez * ez, r = sqrt(r2), r3 = r2 * r;
      v.phi += s->q[j] / r;
      v.g[0] += s->q[j] * ex / r3;
      v.g[1] += s->q[j] * ey / r3;
      v.g[2] += s->q[j] * ez / r3;
    }
  }
  *phi = v.phi;
  g[0] = v.g[0];
  g[1] = v.g[1];
  g[2] = v.g[2];
  return OR_OK;
}

/* Single-ion energy U(x) = l_B [q phi(x) + q'(x) phi(x'(x)) + q q'(x)/|x - x'(x)|]
   on the pre-move tree with the ion and its image excluded, and its gradient.
   The image rule x' = R^2 x/|x|^2, q' = alpha q R/|x| gives
   grad q' = -q' x/|x|^2, d x'/d x = (R^2/|x|^2)(I - 2 x x^T/|x|^2) and a pair
   term alpha q^2 R/(|x|^2 - R^2). */
static int or_ion_energy(or_sys* s, int64_t i, const double x[3], double* U, double gU[3]) {
  int64_t excl[2] = {i, img_index(s, i)};
  int n_excl = s->P.images ? 2 : 1;
  double q = s->q[i], phi, g[3];
  or_phi_grad(s, x, n_excl, excl, &phi, g);
  double u = q * phi;
  double gu[3] = {q * g[0], q * g[1], q * g[2]};
  if (s->P.images) {
    double xi[3], qi;
    if (or_image_of(s, x, q, xi, &qi) != OR_OK) return OR_EDOMAIN;
    double phi2, g2[3];
    or_phi_grad(s, xi, n_excl, excl, &phi2, g2);
    double R = s->P.image_R, al = s->P.image_alpha;
    double r2 = (x[0] * x[0] + x[1] * x[1]) + x[2] * x[2];
    u += qi * phi2;
    double dx[3] = {x[0] - xi[0], x[1] - xi[1], x[2] - xi[2]};
    u += q * qi / sqrt((dx[0] * dx[0] + dx[1] * dx[1]) + dx[2] * dx[2]);
    double f = R * R / r2;
    double xg = (x[0] * g2[0] + x[1] * g2[1]) + x[2] * g2[2];
    double pden = r2 - R * R;
    for (int c = 0; c < 3; ++c) {
      double jt = f * (g2[c] - 2.0 * x[c] * xg / r2); /* (dx'/dx)^T grad phi(x') */
      gu[c] += qi * jt - phi2 * qi * x[c] / r2;     /* q' J^T grad phi(x') + phi(x') grad q' */
      gu[c] += -al * q * q * R * 2.0 * x[c] / (pden * pden);
    }
  }
  *U = s->P.lB * u;
  for (int c = 0; c < 3; ++c) gU[c] = s->P.lB * gu[c];
  return OR_OK;
}

/* Metropolis-adjusted Langevin single-ion moves: b = a - tau beta grad U(a) +
   sqrt(2 tau) xi (xi from Box-Muller on Philox block (m, replica, 2)), accepted
   iff ln alpha <= -beta (U(b) - U(a)) - |a - b + tau beta grad U(b)|^2/(4 tau)
   + |b - a + tau beta grad U(a)|^2/(4 tau). */
int or_mala_run(or_sys* s, uint64_t seed, uint32_t replica, uint64_t m0, int64_t n_moves, double tau,
                or_record* recs, int64_t* n_accepted) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  int64_t acc = 0;
  if (n_moves > 0 && s->n_mob < 1) return OR_EINVAL;
  if (s->P.p + 1 > OR_PMAX) return OR_EINVAL;
  const double two_pi = 6.283185307179586;
  for (int64_t t = 0; t < n_moves; ++t) {
    uint64_t mm = m0 + (uint64_t)t;
    uint32_t ctr[4] = {(uint32_t)mm, (uint32_t)(mm >> 32), replica, 0u};
    uint32_t u[4], v[4], w[4];
    or_philox4x32_10(ctr, key, u);
    ctr[3] = 1u;
    or_philox4x32_10(ctr, key, v);
    ctr[3] = 2u;
    or_philox4x32_10(ctr, key, w);
    int64_t i = (int64_t)(((uint64_t)u[0] * (uint64_t)s->n_mob) >> 32);
    double un[4];
    for (int k = 0; k < 4; ++k) un[k] = ((double)w[k] + 0.5) * 0x1p-32;
    double rad0 = sqrt(-2.0 * log(un[0])), rad1 = sqrt(-2.0 * log(un[2]));
    double xi[3] = {rad0 * cos(two_pi * un[1]), rad0 * sin(two_pi * un[1]), rad1 * cos(two_pi * un[3])};
    double a[3] = {s->x[3 * i], s->x[3 * i + 1], s->x[3 * i + 2]};
    double Ua, ga[3], b[3];
    or_record r;
    memset(&r, 0, sizeof r);
    r.i = i;
    double alpha = ((double)v[0] + 0.5) * 0x1p-32;
    r.log_alpha = log(alpha);
    or_ion_energy(s, i, a, &Ua, ga);
    double sd = sqrt(2.0 * tau), tb = tau * s->P.beta;
    for (int c = 0; c < 3; ++c) b[c] = (a[c] - tb * ga[c]) + sd * xi[c];
    memcpy(r.r_new, b, sizeof b);
    or_move mv;
    int st = prepare_move(s, i, b, &mv);
    if (st == OR_EDOMAIN) {
      r.outcome = OR_REJECT_DOMAIN;
    } else if (st == OR_EOVERLAP) {
      r.outcome = OR_REJECT_OVERLAP;
    } else {
      double Ub, gb[3];
      or_ion_energy(s, i, b, &Ub, gb);
      double dE = Ub - Ua;
      double fwd = 0.0, rev = 0.0;
      for (int c = 0; c < 3; ++c) {
        double f = b[c] - a[c] + tb * ga[c];
        double g = a[c] - b[c] + tb * gb[c];
        fwd += f * f;
        rev += g * g;
      }
      double lacc = -s->P.beta * dE - rev / (4.0 * tau) + fwd / (4.0 * tau);
      r.dE = dE;
      r.flagged = fabs(lacc - r.log_alpha) < 1e-6;
      if (!(r.log_alpha <= lacc)) {
        r.outcome = OR_REJECT_ENERGY;
      } else if (or_capacity_violation(s, i, b)) {
        r.outcome = OR_REJECT_CAPACITY;
      } else {
        or_commit_move(s, i, b);
        r.outcome = OR_ACCEPT;
        acc++;
      }
    }
    if (recs) recs[t] = r;
  }
  if (n_accepted) *n_accepted = acc;
  return OR_OK;
}

int or_ion_energy_grad(or_sys* s, int64_t i, const double x[3], double* U, double gU[3]) {
  if (i < 0 || i >= s->n_mob) return OR_EINVAL;
  return or_ion_energy(s, i, x, U, gU);
}

/* ------------------------------------------------------------------------- */
/* Radial distribution and integrated charge of Sec. 4 (Fig. 6). */
int or_radial_counts(const or_sys* s, int nbins, double r_lo, double r_hi, int64_t* counts, double* charge) {
  if (nbins < 1 || !(r_hi > r_lo)) return OR_EINVAL;
  double w = (r_hi - r_lo) / (double)nbins;
  for (int64_t i = 0; i < s->n_mob; ++i) {
    double x = s->x[3 * i], y = s->x[3 * i + 1], z = s->x[3 * i + 2];
    double r = sqrt((x * x + y * y) + z * z);
    if (!(r >= r_lo && r < r_hi)) continue;
    double t = floor((r - r_lo) / w);
    if (!(t >= 0.0 && t < (double)nbins)) continue;
    counts[(int)t] += 1;
    charge[(int)t] += s->q[i];
  }
  return OR_OK;
}

int or_radial_profiles(int nbins, double r_lo, double r_hi, const int64_t* counts, const double* charge,
                       int64_t n_samples, double q_fixed, double* r_mid, double* g, double* r_out, double* Q) {
  if (nbins < 1 || !(r_hi > r_lo) || n_samples < 1) return OR_EINVAL;
  const double pi = 3.14159265358979323846;
  double w = (r_hi - r_lo) / (double)nbins;
  double total = 0.0, q = q_fixed;
  for (int k = 0; k < nbins; ++k) {
    double a = r_lo + k * w, b = r_lo + (k + 1) * w;
    double vol = 4.0 / 3.0 * pi * (b * b * b - a * a * a);
    g[k] = ((double)counts[k] / (double)n_samples) / vol; /* mean density of bin k */
    total += g[k];
    q += charge[k] / (double)n_samples;
    r_mid[k] = 0.5 * (a + b);
    r_out[k] = b;
    Q[k] = q;
  }
  for (int k = 0; k < nbins; ++k) g[k] = total > 0.0 ? g[k] / total : 0.0;
  return OR_OK;
}
