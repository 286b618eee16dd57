/*
 * bhmc.h -- C-ABI of the GB300 Barnes-Hut octree treecode for Metropolis Monte
 * Carlo of charged systems (Z. Gan, Z. Xu, "Efficient implementation of the
 * Barnes-Hut octree algorithm for Monte Carlo simulations of charged systems",
 * Sci. China Math. 2013).
 *
 * Conventions shared by every call:
 *  - Every call returns a bhmc_status; nothing aborts and no C++ exception
 *    crosses this boundary.
 *  - A context owns all its device state (charges, octree, moments, pools).
 *    Caller buffers passed in are copied; the caller keeps their ownership.
 *  - Work is ordered on the CUDA stream given at creation.  Calls that return a
 *    host value synchronise that stream.
 *  - A failure inside a kernel (pool exhausted, traversal stack overflow) is
 *    recorded in the context and returned by the call that launched it and by
 *    every later call (BHMC_ESTATE) until the context is destroyed.
 *  - Charge indexing: [0, n_mobile) mobile ions, [n_mobile, n_mobile+n_fixed)
 *    fixed charges, then (with images) the image of ion i at n_mobile+n_fixed+i.
 *  - Lengths are in the unit of l_B; energies are beta*V (units of k_B T).
 */
#ifndef BHMC_H
#define BHMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BHMC_OK = 0,
  BHMC_EINVAL = 1,      /* invalid argument or parameter */
  BHMC_EDOMAIN = 2,     /* a position lies outside the root cube */
  BHMC_EOVERLAP = 3,    /* a position violates the confinement shell */
  BHMC_ENOMEM = 4,      /* device or host allocation failed */
  BHMC_ENOMEM_POOL = 5, /* the node pool of a context is exhausted */
  BHMC_ECUDA = 6,       /* a CUDA runtime call failed */
  BHMC_ETIMEOUT = 7,    /* a bounded device loop ran out of iterations */
  BHMC_ESTATE = 8,      /* the context holds an earlier device error */
  BHMC_ECAPACITY = 9,   /* a depth-Dmax cell would hold more than C charges */
  BHMC_ESTACK = 10,     /* a traversal stack overflowed */
  BHMC_ESCRATCH = 11,   /* problem larger than a call's fixed scratch allows */
  BHMC_ENONFINITE = 12  /* a trial's energy difference was not finite (the FP32 expansion
                           overflowed: use BHMC_PREC_F64 or a lower order); the trial is
                           rejected and the chain stops at the next move */
} bhmc_status;

enum { BHMC_PREC_F32 = 0, BHMC_PREC_F64 = 1 };   /* traversal arithmetic */
enum { BHMC_LAYOUT_SOA = 0, BHMC_LAYOUT_AOS = 1 }; /* FP32 moment layout */
enum { BHMC_HOST_PTRS = 0, BHMC_DEVICE_PTRS = 1 }; /* flags: where caller arrays live */

/* Outcome of one Metropolis trial move (Sec. 2 of the paper, step 2). */
enum {
  BHMC_ACCEPT = 0,
  BHMC_REJECT_ENERGY = 1,   /* alpha > exp(-beta dE) */
  BHMC_REJECT_DOMAIN = 2,   /* trial position (or its image) outside the root cube */
  BHMC_REJECT_OVERLAP = 3,  /* trial position outside the confinement shell */
  BHMC_REJECT_CAPACITY = 4  /* would overfill a depth-Dmax cell */
};

/* Parameters of a system.  Cites: l_B and beta, Eq. (1.1)/(2.1); theta, p and
   N0, Sec. 3.2 and Eq. (3.3); the root cube, Sec. 3.2; the cell model, Sec. 4. */
typedef struct {
  double lB;          /* Bjerrum length (> 0) */
  double beta;        /* inverse temperature of the Metropolis rule (>= 0) */
  double theta;       /* MAC: multipole iff rho_A/|r_A - x| <= theta, 0 <= theta < 1 */
  int32_t p;          /* Taylor truncation order, 0..10.  With FP32 traversal the order-p terms
                         T_n overflow for accepted clusters closer than about 2e-3 length
                         units at p = 10 (1e-5 at p = 6); BHMC_PREC_F64 has no such limit */
  int32_t N0;         /* minimum expansion number (>= 0) */
  int32_t C;          /* leaf capacity, 2..32: a cluster holding more than C charges splits (more
                         than 0 with fixed_depth); no depth-Dmax cell may hold more than C */
  int32_t Dmax;       /* deepest level, 1..20 */
  double root_lo[3];  /* lower corner of the root cube, a multiple of side/2^Dmax */
  double root_side;   /* side of the root cube, a power of two */
  int32_t shell;      /* 1: mobile ions confined to shell_rmin <= |r| <= shell_rmax */
  double shell_rmin, shell_rmax;
  int32_t images;     /* 1: each mobile ion carries an image at R^2 r/|r|^2, charge alpha q R/|r| */
  double image_R, image_alpha;
  int32_t precision;  /* BHMC_PREC_F32 (FP32 traversal, FP64 moments) or BHMC_PREC_F64 (all FP64) */
  int32_t warps;      /* warps cooperating on one move: 1, 2, 4 or 8 */
  int32_t layout;     /* BHMC_LAYOUT_SOA or BHMC_LAYOUT_AOS for the FP32 moment mirror */
  double node_factor; /* node pool = 64 + node_factor * charges (0 selects 1 + max(1, 8/C), or
                         8 (Dmax - floor(log8 charges) + 1) with fixed_depth) */
  double hard_core;   /* common diameter tau of the mobile ions (Eq. 2.1: the pair potential is
                         infinite for r_ij <= tau); a trial position within tau of another mobile
                         ion is rejected (BHMC_REJECT_OVERLAP); 0 disables.  Images and fixed
                         charges carry no hard core (the macroion's is the shell). */
  int32_t fixed_depth; /* 1: the fixed-level tree of Sec. 3.2 with L_max = Dmax (every non-empty
                          cluster above Dmax is bisected, so all charges sit in depth-Dmax
                          leaves); 0: the adaptive tree of leaf capacity C */
  int32_t fixed_direct; /* 1: the fixed charges (Sec. 4: the macroion, fixed at the cell centre)
                           stay out of the tree and interact exactly: every potential evaluated
                           by the treecode adds their terms q_f / |x - r_f| in FP64, and the
                           potential at a fixed charge is the exact sum over all other charges.
                           0: fixed charges are ordinary tree charges */
  int32_t round_limit;  /* iteration budget of the bounded device loops (traversal rounds of a
                           trial move, stack pops of one warp in the energy and force passes);
                           0 selects the defaults (2^22 and 2^24).  A loop that runs out stops
                           and its call returns BHMC_ETIMEOUT; inside a chain (step calls) the
                           error is also latched, and later calls return BHMC_ESTATE.  A small
                           value exercises that path without any device fault */
} bhmc_params;

typedef struct bhmc_ctx bhmc_ctx;
typedef struct bhmc_batch bhmc_batch;

/* Interaction-list counters of one evaluation (equal to the oracle's). */
typedef struct {
  int64_t visited;  /* (cluster, evaluation point) pairs examined */
  int64_t accepted; /* pairs evaluated by the multipole approximation */
  int64_t pairs;    /* particle-particle direct terms */
  int64_t mac_fp64; /* MAC decisions settled by the exact FP64 test */
} bhmc_counters;

/* One trial move of a Monte Carlo run. */
typedef struct {
  int64_t i;        /* chosen mobile ion */
  double r_new[3];  /* trial position */
  double dE;        /* energy difference (0 if rejected before evaluation) */
  int32_t outcome;  /* BHMC_ACCEPT or BHMC_REJECT_* */
  int32_t flagged;  /* 1 if |beta dE + ln alpha| < 1e-6 (decision near the threshold) */
} bhmc_move_record;

typedef struct {
  int64_t moves, accepted, rej_energy, rej_domain, rej_overlap, rej_capacity, flagged;
  double energy;    /* running energy: sum of accepted dE since creation or bhmc_set_energy */
} bhmc_mc_stats;

const char* bhmc_status_string(bhmc_status s);

/* Build the octree of n_mobile + n_fixed charges (Sec. 3.2: the root cube is
   bisected recursively; a cluster holding more than C charges is split until
   level Dmax) and the FP64 moments M_A^n = sum_j q_j (r_j - r_A)^n of Eq. (3.3).
   q[n], xyz[3n] (x,y,z interleaved), host or device memory per `flags`,
   copied.  cuda_stream: a cudaStream_t or NULL for the default stream.
   Errors: EINVAL (parameters), EDOMAIN (charge or image outside the root),
   EOVERLAP (ion outside the shell), ECAPACITY, ENOMEM, ECUDA. */
bhmc_status bhmc_create(const bhmc_params* params, int64_t n_mobile, int64_t n_fixed,
                        const double* q, const double* xyz, int32_t flags, void* cuda_stream,
                        bhmc_ctx** out);
bhmc_status bhmc_destroy(bhmc_ctx* ctx);

/* Number of charges in the tree (ions, fixed charges and images). */
bhmc_status bhmc_n_charges(const bhmc_ctx* ctx, int64_t* n);
/* Copy current charges and positions (xyz interleaved) to host or device buffers. */
bhmc_status bhmc_get_charges(bhmc_ctx* ctx, double* q, double* xyz, int32_t flags);
/* Positions only (n_charges x 3, interleaved), host or device buffer per flags. */
bhmc_status bhmc_get_positions(bhmc_ctx* ctx, double* xyz, int32_t flags);
/* Interaction-list counters of the last successful bhmc_delta_energy or
   bhmc_energy_counters call on this context (zeros before any). */
bhmc_status bhmc_get_counters(bhmc_ctx* ctx, bhmc_counters* out);

/* Energy difference of moving mobile ion i (and its image) to r_new (Sec. 1:
   V_i evaluated before and after the displacement; Sec. 3.2 traversal with the
   multipole approximation of Eq. (3.3)); the state is not modified.  The moved
   charges are excluded from the pre-move tree.  Returns EDOMAIN/EOVERLAP when
   the trial position would be rejected before any evaluation.  counters may be
   NULL. */
bhmc_status bhmc_delta_energy(bhmc_ctx* ctx, int64_t i, const double r_new[3], double* dE,
                              bhmc_counters* counters);

/* Local adjustment of Sec. 3.3 for a move of ion i (and its image) to r_new,
   applied unconditionally: remove from the old leaf (swap with the last slot),
   insert into the new one, update counts and FP64 moments on both ancestor
   paths, merge/split clusters so the tree stays the canonical tree of the
   particle set.  Errors: EDOMAIN, EOVERLAP, ECAPACITY (state unchanged),
   ENOMEM_POOL. */
bhmc_status bhmc_commit_move(bhmc_ctx* ctx, int64_t i, const double r_new[3]);

/* n_moves Metropolis trials (Sec. 2), one kernel launch per trial.  Trial m
   uses Philox4x32-10 with key (seed) and counter (m, 0, 0) for the ion index
   and displacement (uniform in [-step/2, step/2)^3) and counter (m, 0, 1) for
   alpha; m runs from move0.  stats must not be NULL; records (host, n_moves
   entries) may be NULL. */
bhmc_status bhmc_step_mc(bhmc_ctx* ctx, uint64_t n_moves, double step, uint64_t seed,
                         uint64_t move0, bhmc_mc_stats* stats, bhmc_move_record* records);

/* The same chain as bhmc_step_mc (same trials, outcomes, records and final
   state), in one launch of a thread-block cluster of `proposals` CTAs
   (1..BHMC_MAX_PROPOSALS): each step evaluates trials m .. m+proposals-1
   concurrently against the current tree and keeps them up to the first
   acceptance, which is committed; a trial evaluated while every earlier trial
   of its step was rejected sees the tree the sequential chain would see
   (Sec. 2: a rejected move leaves the configuration unchanged).  Speeds up a
   single chain by up to 1/acceptance.  EINVAL for proposals outside the range. */
#define BHMC_MAX_PROPOSALS 8
bhmc_status bhmc_step_mc_spec(bhmc_ctx* ctx, uint64_t n_moves, double step, uint64_t seed,
                              uint64_t move0, int32_t proposals, bhmc_mc_stats* stats,
                              bhmc_move_record* records);

/* n_moves Metropolis-adjusted Langevin single-ion trials, one launch each: the
   ion's energy U(x) (the potential of the tree without the ion and its image,
   at the ion and at its image, plus the pair term) and its gradient at the
   current position a come from one traversal; the trial position is
   b = a - tau beta grad U(a) + sqrt(2 tau) xi with xi normal (Box-Muller on
   Philox counter (m, 0, 2)); a second traversal gives U(b) and grad U(b); the
   trial is accepted iff ln alpha <= -beta (U(b) - U(a)) - |a - b + tau beta
   grad U(b)|^2 / (4 tau) + |b - a + tau beta grad U(a)|^2 / (4 tau).  Not in the
   paper (its proposals are uniform displacements, Sec. 2). */
bhmc_status bhmc_step_mala(bhmc_ctx* ctx, uint64_t n_moves, double tau, uint64_t seed, uint64_t move0,
                           bhmc_mc_stats* stats, bhmc_move_record* records);

/* Radial distribution of the mobile ions (Sec. 4: RDF g(r) and ICDF Q(r) of
   the double layer): for every mobile ion with r_lo <= r < r_hi, r = sqrt((x x
   + y y) + z z) in FP64, bin k = floor((r - r_lo) / ((r_hi - r_lo) / nbins)),
   adds 1 to counts[k] and its charge to charge[k] (host arrays of nbins,
   accumulated, so that calls between steps average over the chain).
   BHMC_EINVAL for nbins outside [1, 2^24] or r_hi <= r_lo.  Not a call of the
   paper; it measures its Fig. 6 quantities. */
bhmc_status bhmc_radial_counts(bhmc_ctx* ctx, int32_t nbins, double r_lo, double r_hi, int64_t* counts,
                               double* charge);

/* Radial sampling inside the chains (Sec. 4, Fig. 6: the RDF and ICDF are
   averages over the configurations of the Markov chain).  With nbins > 0 the
   context keeps a running histogram of its mobile ions (bins as in
   bhmc_radial_counts, built from the current configuration by this call and
   updated by every committed move on the device), and every chain call
   (bhmc_step_mc, bhmc_step_mc_spec, bhmc_step_mala) adds it to device
   accumulators after each move m with (m + 1) % every == 0 (m the absolute
   move index, so the samples do not depend on how the chain is split into
   calls).  The accumulators start at zero here; nbins = 0 switches sampling
   off.  EINVAL for nbins outside [0, 2^20], every < 0, r_hi <= r_lo, or a
   replica of a batch (use bhmc_batch_set_radial_sampling). */
bhmc_status bhmc_set_radial_sampling(bhmc_ctx* ctx, int32_t nbins, double r_lo, double r_hi, int64_t every);
/* The accumulated samples: counts[nbins] and charge[nbins] (host; the sums of
   the running histogram over the samples) and the number of samples.
   BHMC_ESTATE if sampling is off. */
bhmc_status bhmc_get_radial_samples(bhmc_ctx* ctx, int64_t* counts, double* charge, int64_t* n_samples);
/* RDF and ICDF of Sec. 4 from accumulated counts (host arithmetic only, no
   device call): <N_k> = counts[k] / n_samples, V_k = (4/3) pi (r_{k+1}^3 -
   r_k^3) with r_k = r_lo + k (r_hi - r_lo) / nbins;
   g[k] = (<N_k>/V_k) / sum_j (<N_j>/V_j) (the bins normalised to sum one);
   Q[k] = q_fixed + sum_{j <= k} charge[j] / n_samples, the charge inside the
   outer edge r_out[k] of bin k (Q(a) = Q_M and Q(R_cell) = 0 for the
   neutral cell of Sec. 4); r_mid[k] is the bin centre.  All arrays have nbins
   entries.  EINVAL for nbins < 1, r_hi <= r_lo or n_samples < 1. */
bhmc_status bhmc_radial_profiles(int32_t nbins, double r_lo, double r_hi, const int64_t* counts,
                                 const double* charge, int64_t n_samples, double q_fixed, double* r_mid, double* g,
                                 double* r_out, double* Q);

/* Running energy (sum of accepted dE since creation, or rebased by set). */
bhmc_status bhmc_get_energy(bhmc_ctx* ctx, double* E);
bhmc_status bhmc_set_energy(bhmc_ctx* ctx, double E);

/* Total treecode energy E = (1/2) l_B sum_i q_i phi_tree(r_i), every charge
   excluded from its own sum (Eq. 1.1 evaluated by the Sec. 3.2 traversal). */
bhmc_status bhmc_energy(bhmc_ctx* ctx, double* E);
/* bhmc_energy plus the interaction-list counters summed over every target
   (visited clusters, multipole evaluations, direct pairs; mac_fp64 is 0): the
   per-target counts are those of the Sec. 3.2 traversal at r_j with j excluded. */
bhmc_status bhmc_energy_counters(bhmc_ctx* ctx, double* E, bhmc_counters* total);
/* Treecode potential of every charge, phi_j = sum over the tree minus j of
   q_k / |r_k - r_j| (the traversal of Sec. 3.2 at r_j), into phi[n_charges]
   (host or device memory per flags).  The same pass as bhmc_energy. */
bhmc_status bhmc_potentials(bhmc_ctx* ctx, double* phi, int32_t flags);
/* Gradient of the total treecode energy with every MAC decision held fixed
   (the adjoint of the Sec. 3.2 traversal and of the moments of Eq. 3.3):
   dEdr[3k..3k+2] = dE/dr_k (forces are -dEdr), dEdq[k] = dE/dq_k for every
   charge (ions, fixed charges and images as independent charges); host or
   device buffers per flags.  Scratch of about (8 + 8K nodes/charge) doubles per
   charge is allocated for the call. */
bhmc_status bhmc_forces(bhmc_ctx* ctx, double* dEdr, double* dEdq, int32_t flags);
/* Total energy by direct O(N^2) summation of Eq. (1.1) on the GPU (FP64). */
bhmc_status bhmc_energy_direct(bhmc_ctx* ctx, double* E);

/* Tree export for parity checks.  rows[4*k..4*k+3] = (depth, Morton key with a
   leading 1 bit, is_leaf, count) in depth-first order (children in octant
   order); members receives every leaf's charge indices (sorted) in row order.
   moments (may be NULL) receives the FP64 moments, K(p) per row.  *n_rows is
   the number of rows written.  EINVAL if a buffer is too small. */
bhmc_status bhmc_export_tree(bhmc_ctx* ctx, int64_t* rows, int64_t max_rows, int64_t* members,
                             int64_t max_members, double* moments, int64_t* n_rows);

/* Direct-sum total energy E = (1/2) l_B sum_{i != j} q_i q_j / r_ij (FP64) of
   n charges, for callers that cannot call cudaMalloc when they need it:
   applications that reserve their device memory up front and give libraries
   only pre-allocated buffers, and loops that must not take the device-wide
   synchronisation an allocation can cause.  The paper has no counterpart; it
   is the variant of bhmc_energy_direct whose scratch is a fixed 32 KiB
   __device__ array inside the library (held by every device that loads the
   library until the process exits).  q[n], xyz[3n] (x,y,z interleaved) and
   E[1] are DEVICE pointers owned by the caller; E is written on cuda_stream
   (no host synchronisation).  n <= 1048576, else BHMC_ESCRATCH before any
   launch; n < 1 or a null pointer: BHMC_EINVAL.  The call allocates nothing
   (no cudaMalloc, cudaFree or allocating library routine).  The first call in
   a CUDA context (per device, and again after a device reset) looks up the
   scratch's device address with that context current; make that first call
   before any stream capture.  All calls share the scratch, so calls whose
   kernels overlap on one device race on it; each call writes every scratch
   entry it reads, so nothing needs clearing between calls. */
bhmc_status bhmc_energy_direct_noalloc(int64_t n, const double* q, const double* xyz, double lB,
                                       double* E, void* cuda_stream);

/* ---- batches of independent replicas (one octree each) ---- */

/* n_rep systems sharing one parameter set; replica r has n_mobile[r] ions and
   n_fixed[r] fixed charges with arrays q[r], xyz[r]. */
bhmc_status bhmc_batch_create(int32_t n_rep, const bhmc_params* params, const int64_t* n_mobile,
                              const int64_t* n_fixed, const double* const* q,
                              const double* const* xyz, int32_t flags, void* cuda_stream,
                              bhmc_batch** out);
bhmc_status bhmc_batch_destroy(bhmc_batch* batch);
/* Borrowed context of replica r (valid until the batch is destroyed; do not destroy it). */
bhmc_status bhmc_batch_replica(bhmc_batch* batch, int32_t r, bhmc_ctx** ctx);
/* bhmc_set_radial_sampling for every replica of the batch (the batched chain
   calls then sample as the single-context calls do). */
bhmc_status bhmc_batch_set_radial_sampling(bhmc_batch* batch, int32_t nbins, double r_lo, double r_hi,
                                           int64_t every);
/* Per replica: counts[r * nbins + k], charge[r * nbins + k], n_samples[r]. */
bhmc_status bhmc_batch_get_radial_samples(bhmc_batch* batch, int64_t* counts, double* charge,
                                          int64_t* n_samples);
/* bhmc_radial_counts summed over every replica of the batch. */
bhmc_status bhmc_batch_radial_counts(bhmc_batch* B, int32_t nbins, double r_lo, double r_hi, int64_t* counts,
                                     double* charge);

/* n_moves Metropolis trials on every replica in ONE persistent kernel launch,
   replayed from a CUDA graph.  Replica r uses key seeds[r] and counter
   (m, r, tag).  stats: n_rep entries (may be NULL). */
bhmc_status bhmc_batch_step_mc(bhmc_batch* batch, uint64_t n_moves, double step,
                               const uint64_t* seeds, uint64_t move0, bhmc_mc_stats* stats);

/* bhmc_batch_step_mc with one record per trial move: records[r * n_moves + t]
   (host, n_rep x n_moves, replica-major) receives move t of replica r (the
   same fields as bhmc_step_mc's records).  The records buffer is allocated on
   the device for the call.  EINVAL if records is NULL. */
bhmc_status bhmc_batch_step_mc_records(bhmc_batch* batch, uint64_t n_moves, double step,
                                       const uint64_t* seeds, uint64_t move0, bhmc_mc_stats* stats,
                                       bhmc_move_record* records);

/* The same chains as bhmc_batch_step_mc, each on its own thread-block cluster
   of `proposals` CTAs evaluating that many trials per step (as
   bhmc_step_mc_spec), all replicas in one launch of replicas x proposals CTAs.
   For batches too small to fill the GPU with one CTA per replica.  EINVAL for
   proposals outside 1..BHMC_MAX_PROPOSALS. */
bhmc_status bhmc_batch_step_mc_spec(bhmc_batch* batch, uint64_t n_moves, double step,
                                    const uint64_t* seeds, uint64_t move0, int32_t proposals,
                                    bhmc_mc_stats* stats);

#ifdef __cplusplus
}
#endif
#endif
