/*
 * bhmc_oracle.h -- plain FP64 CPU oracle of the Barnes-Hut octree Monte Carlo
 * method for charged systems (Gan & Xu, Sci. China Math. 2013).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg load this library.  It shares no code, no
 * header and no constant with the CUDA path, and the CUDA path never calls it.
 *
 * Everything is double precision, single threaded, compiled without FMA
 * contraction or fast-math, so that every floating-point operation is the one
 * written in the source.
 */
#ifndef BHMC_ORACLE_H
#define BHMC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_PMAX 10 /* highest multipole order supported (Sec. 4 sweeps p = 0..10) */
#define OR_DMAX 20 /* deepest tree level (60-bit Morton keys) */

/* Status codes (same meaning as the library's, separate definitions). */
enum {
  OR_OK = 0,
  OR_EINVAL = 1,
  OR_EDOMAIN = 2,   /* position outside the root cube */
  OR_EOVERLAP = 3,  /* position violates the confinement shell */
  OR_ENOMEM = 4,
  OR_ECAPACITY = 9  /* a depth-Dmax cell would hold more than C charges */
};

/* Move outcomes of one Metropolis trial (Sec. 2, steps of the MC algorithm). */
enum {
  OR_ACCEPT = 0,
  OR_REJECT_ENERGY = 1,
  OR_REJECT_DOMAIN = 2,
  OR_REJECT_OVERLAP = 3,
  OR_REJECT_CAPACITY = 4
};

typedef struct {
  double lB;        /* Bjerrum length, Eq. (1.1) */
  double beta;      /* inverse thermal energy, Eq. (2.1) */
  double theta;     /* opening parameter of the MAC rho_A / r_{i,A} <= theta, Sec. 3.2 */
  int32_t p;        /* truncation order of the Taylor expansion, Eq. (3.3) */
  int32_t N0;       /* minimum expansion number N_0, Sec. 3.2 */
  int32_t C;        /* leaf capacity: a node splits when it holds more than C charges
                       (more than 0 with fixed_depth); no depth-Dmax leaf holds more */
  int32_t Dmax;     /* deepest level */
  double root_lo[3];/* lower corner of the root cube (Sec. 3.2 root cluster) */
  double root_side; /* side of the root cube, a power of two */
  int32_t shell;    /* 1: mobile ions confined to rmin <= |r| <= rmax (Sec. 4 cell model) */
  double shell_rmin, shell_rmax;
  int32_t images;   /* 1: every mobile ion carries a point image that moves with it */
  double image_R;   /* image position R^2 r / |r|^2 */
  double image_alpha; /* image charge alpha * q * R / |r| */
  double hard_core; /* common diameter tau of the mobile ions (Eq. 2.1), 0: none */
  int32_t fixed_depth; /* 1: the Sec. 3.2 tree of fixed level L_max = Dmax: every
                          non-empty cluster above Dmax splits, leaves are at Dmax */
  int32_t fixed_direct; /* 1: the fixed charges (the macroion of Sec. 4, fixed at the
                           cell centre) stay out of the tree; every potential adds their
                           exact terms q_f / |x - r_f|, and the potential at a fixed
                           charge is the exact sum over all other charges */
} or_params;

typedef struct or_sys or_sys;

/* One treecode evaluation of the potential at a point (Sec. 3.2). */
typedef struct {
  double phi;      /* sum_j q_j / |r_j - x| over the tree minus the excluded set, treecode */
  double abs_sum;  /* sum of |term| over the interaction list (multipole: sum_n |T_n M_n|) */
  double bound;    /* truncation bound of Eq. (3.4) summed over accepted clusters (per-order form) */
  int64_t visited; /* clusters examined */
  int64_t accepted;/* clusters evaluated by the multipole approximation */
  int64_t pairs;   /* particle-particle direct terms */
  int64_t mac_near;/* accepted/rejected MAC decisions within 2^-17 relative of the threshold */
} or_eval;

typedef struct {
  double dE;       /* beta-free energy difference l_B * (...) of the trial move */
  double abs_sum;  /* l_B * sum over the four evaluations of |weight| * abs_sum */
  double bound;    /* l_B * sum of |weight| * bound */
  int64_t visited, accepted, pairs;
  int32_t status;  /* OR_OK, OR_EDOMAIN or OR_EOVERLAP */
} or_dE;

typedef struct {
  int64_t i;        /* chosen mobile ion */
  double r_new[3];  /* trial position */
  double dE;        /* treecode energy difference (0 when rejected before evaluation) */
  double abs_sum;   /* conditioning sum of dE */
  double log_alpha; /* ln of the uniform number compared with exp(-beta dE) */
  int32_t outcome;  /* OR_ACCEPT, OR_REJECT_* */
  int32_t flagged;  /* 1 if |beta dE + ln alpha| < 1e-6 */
} or_record;

/* ---- primitives ---- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
int or_nterms(int p);
int or_term_index(int n1, int n2, int n3);
/* T_n(R) for ||n|| <= p in graded order (recurrence of Sec. 3.1). */
int or_taylor(int p, const double R[3], double* T);
/* l_B * sum_{i<j} q_i q_j / r_ij over n charges (Eq. 1.1); xyz is n x 3. */
double or_direct_energy_raw(int64_t n, const double* q, const double* xyz, double lB);

/* ---- system ---- */
/* n_mob mobile ions first, then n_fix fixed charges; xyz is n x 3.  Images are
   appended internally (charge index n_mob + n_fix + i is the image of ion i). */
or_sys* or_create(const or_params* P, int64_t n_mob, int64_t n_fix, const double* q,
                  const double* xyz, int* status);
void or_destroy(or_sys* s);
/* 1: accumulate the Eq. (3.4) truncation bound during traversals (costs O(N_A) per accepted cluster). */
void or_set_bound(or_sys* s, int on);
int64_t or_n_charges(const or_sys* s);
void or_get_charges(const or_sys* s, double* q, double* xyz);
int or_image_of(const or_sys* s, const double r[3], double q, double rim[3], double* qim);

/* Potential at x from all charges except the n_excl listed ones (pre-move tree);
   with fixed_direct the fixed charges enter as exact terms (counted in abs_sum,
   not in the interaction-list counters). */
int or_phi(or_sys* s, const double x[3], int n_excl, const int64_t* excl, or_eval* out);
double or_phi_direct(const or_sys* s, const double x[3], int n_excl, const int64_t* excl);

/* Treecode energy difference of moving ion i (and its image) to b; state unchanged. */
int or_delta_energy(or_sys* s, int64_t i, const double b[3], or_dE* out);
int or_delta_energy_direct(const or_sys* s, int64_t i, const double b[3], double* dE);
/* Local adjustment of Sec. 3.3 (applied unconditionally). */
int or_commit_move(or_sys* s, int64_t i, const double b[3]);
/* 1 if moving ion i to b would put more than C charges into one depth-Dmax cell. */
int or_capacity_violation(or_sys* s, int64_t i, const double b[3]);

/* n_moves Metropolis trials (Sec. 2) with the Philox stream key=(seed), counter=(m, replica, tag). */
int or_mc_run(or_sys* s, uint64_t seed, uint32_t replica, uint64_t m0, int64_t n_moves,
              double step, or_record* recs, int64_t* n_accepted);

/* Total energies over all charges (ions, fixed charges, images). */
double or_energy_direct(const or_sys* s);
double or_energy_tree(or_sys* s);
/* V-bar_i = l_B q_i phi_tree(r_i) and V_i = l_B q_i phi_direct(r_i) for every charge (Eq. 4.1);
   with fixed_direct the potential at a fixed charge is exact on both sides. */
int or_potentials(or_sys* s, double* v_tree, double* v_direct);

/* Exact gradient of the total treecode energy with every MAC decision held
   fixed: dEdr (n x 3) = dE/dr_k, dEdq (n) = dE/dq_k for every charge (ions,
   fixed charges and images treated as independent).  Needs p <= OR_PMAX - 1. */
int or_forces(or_sys* s, double* dEdr, double* dEdq);
/* The same adjoint with every term replaced by its magnitude: per component,
   l_B/2 times the sum of |term| over everything that enters dE/dr_k and
   dE/dq_k (target side, direct source side, and the cluster adjoints built
   from |q_i T_n| and pushed down with |monomial derivatives|).  It is the
   conditioning of the forces: rounding errors in these terms are bounded by a
   multiple of it. */
int or_forces_abs(or_sys* s, double* Ar, double* Aq);

/* Potential and its gradient at x from all charges except the listed ones. */
int or_phi_grad(or_sys* s, const double x[3], int n_excl, const int64_t* excl, double* phi, double g[3]);
/* Single-ion energy U(x) (ion i moved to x, image following; pre-move tree with
   both excluded) and its gradient, as used by the Langevin proposals. */
int or_ion_energy_grad(or_sys* s, int64_t i, const double x[3], double* U, double gU[3]);
/* Metropolis-adjusted Langevin single-ion moves (step tau); Philox blocks
   (m, replica, 0) ion index, (m, replica, 1) alpha, (m, replica, 2) normals. */
int or_mala_run(or_sys* s, uint64_t seed, uint32_t replica, uint64_t m0, int64_t n_moves, double tau,
                or_record* recs, int64_t* n_accepted);

/* Radial distribution of the mobile ions (Sec. 4, Fig. 6): for every mobile
   ion, r = sqrt((x x + y y) + z z) and, when r_lo <= r < r_hi, bin
   k = floor((r - r_lo) / w), w = (r_hi - r_lo) / nbins (all FP64, this order),
   counted when 0 <= k < nbins; counts[k] += 1 and charge[k] += q (the arrays
   are added to, not cleared). */
int or_radial_counts(const or_sys* s, int nbins, double r_lo, double r_hi, int64_t* counts, double* charge);
/* RDF g and ICDF Q of Sec. 4 from counts accumulated over n_samples
   configurations: <N_k> = counts[k] / n_samples, V_k = (4/3) pi (r_{k+1}^3 -
   r_k^3) with r_k = r_lo + k w; g_k = (<N_k>/V_k) / sum_j (<N_j>/V_j) (the bins
   normalised to sum one); Q at the outer edge of bin k = q_fixed + sum_{j<=k}
   charge[j] / n_samples.  r_mid, g, r_out and Q have nbins entries. */
int or_radial_profiles(int nbins, double r_lo, double r_hi, const int64_t* counts, const double* charge,
                       int64_t n_samples, double q_fixed, double* r_mid, double* g, double* r_out, double* Q);

/* Tree export: one row per node (depth, key, is_leaf, count); leaf members are
   written consecutively into members (sorted ascending) in node order.  Returns
   the number of nodes, or -1 if a buffer is too small. */
int64_t or_export_tree(const or_sys* s, int64_t* rows, int64_t max_rows, int64_t* members,
                       int64_t max_members);
/* Structural self-check (counts, membership, tracking, canonical shape).  0 = ok. */
int or_check(const or_sys* s);
/* Moments of the node with the given key (or -1): copies K(p) values. */
int or_node_moments(const or_sys* s, int depth, uint64_t key, double* M);
/* Morton key of a point at depth Dmax (comparison descent), 0 if outside the root. */
uint64_t or_point_key(const or_sys* s, const double x[3]);

#ifdef __cplusplus
}
#endif
#endif
