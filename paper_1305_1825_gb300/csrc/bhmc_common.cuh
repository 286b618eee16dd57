// bhmc_common.cuh -- device-side data layout and helpers of the GB300 treecode
// Monte Carlo (Gan & Xu 2013).  Everything here is written for sm_103a.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/bhmc.h"

#define BHMC_MAX_P 10
#define BHMC_MAX_D 20
#ifndef BHMC_MAX_WARPS
#define BHMC_MAX_WARPS 8
#endif
#define BHMC_ENERGY_WARPS 4
#define BHMC_MAX_C 32

namespace bhmc {

__host__ __device__ constexpr int nterms(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }
__host__ __device__ constexpr int pad4(int k) { return (k + 3) & ~3; }
// graded order of multi-indices (k = 0..p; n1 = k..0; n2 = k-n1..0), Eq. (3.3)
__host__ __device__ constexpr int tidx(int n1, int n2, int n3) {
  return (n1 + n2 + n3) * (n1 + n2 + n3 + 1) * (n1 + n2 + n3 + 2) / 6 +
         (n2 + n3) * (n2 + n3 + 1) / 2 + n3;
}

// Device view of one system.  Node storage: 8 contiguous children per group;
// group 0 holds the root at node 0 (nodes 1..7 stay empty).  Per node:
//   nA = {cx, cy, cz, h} (centre and half side, exact dyadic floats),
//   nB = {first_child or -1, count, key_lo, key_hi} (Morton key with a leading 1).
// Leaf slots: node*C + k, sA = {x_hi, y_hi, z_hi, q}, sB = {x_lo, y_lo, z_lo, idx}
// where x = x_hi + x_lo is the FP64 position split into two floats.
struct SysDev {
  int n_mob, n_fix, n_tot;
  int fixed_direct;         // 1: fixed charges outside the tree, exact terms everywhere
  int n_tree;               // charges in the tree: n_tot, or n_tot - n_fix with fixed_direct
  int move_rounds;          // iteration budgets: traversal rounds of a trial move,
  int pass_pops;            // stack pops of one warp in the energy and force passes
  int p, K, Kp, N0, C, Dmax;
  int Cs;                   // split threshold: C, or 0 for the fixed-level tree
  int images, shell, prec, layout;
  double lB, beta, theta2;
  float theta2f, lBf;
  double root_lo[3], root_side;
  double inv_hmin;          // 2^Dmax / side (a power of two)
  int hmin_shift;           // log2(inv_hmin)
  long long root_cell[3];   // root_lo * inv_hmin (integers)
  double rmin, rmax;        // shell radii
  double rmin2, rmax2;      // rmin * rmin, rmax * rmax (FP64 products)
  double img_R, img_alpha;
  double img_R2;            // img_R * img_R
  double hc2;               // hard-core diameter squared (0: none), Eq. (2.1)
  float hc2f;
  // charges
  double *px, *py, *pz, *pq;
  unsigned long long* ckey;
  int* leaf_of;
  int* slot_of;
  int* order;   // charges in the Morton order of the build (spatially coherent targets)
  // nodes
  int node_cap, group_cap;
  float4* nA;
  int4* nB;
  float* M32;   // SoA [K][node_cap] or AoS [node_cap][Kp]
  double* M64;  // [node_cap][K]
  // Evaluation coefficients W_m = sum_n c(n, m) M_n with r^(2k+1) T_n(R) =
  // sum_{|m| = k} c(n, m) R^m, so that sum_{|n| = k} T_n(R) M_n =
  // r^-(2k+1) sum_{|m| = k} W_m R^m (FP32, laid out like M32; FP32 traversal)
  float* W32;
  int* wrow;    // CSR of the map by output term: wrow[K + 1], wcol/wval[nnz]
  int* wcol;
  float* wval;
  float4* sA;
  float4* sB;
  int* pool;    // pool[0] = next unused group, pool[1] = number of free groups
  int* free_list;
  // state
  double* energy;
  int* err;
  // Radial sampling of the mobile ions during the chains (Sec. 4, Fig. 6;
  // rdf_nbins = 0: off): a running histogram of the current configuration,
  // kept by every committed move, is added to the accumulators after every
  // rdf_every-th move (absolute move index).
  int rdf_nbins;
  long long rdf_every;
  double rdf_lo, rdf_hi, rdf_w;
  unsigned long long* rdf_run;   // [nbins] current counts
  double* rdf_runq;              // [nbins] current charge
  unsigned long long* rdf_acc;   // [nbins] summed over the samples
  double* rdf_accq;              // [nbins]
  unsigned long long* rdf_nsamp; // [1]
};

struct MoveRec;

// Arguments of one batched launch (device memory).
struct BatchArgs {
  unsigned long long n_moves, move0;
  double step;
  const unsigned long long* seeds;
  const int* order;  // replicas in the order blocks take them (largest first)
  MoveRec* recs;     // null, or n_rep x n_moves per-move records (replica-major)
  int* errs;         // null, or n_rep: each replica's error word when its chain ends
  // Which block runs which replica.  A block runs a replica's chain after
  // setting its claim flag; blocks without one take entries of `order` from
  // `cursor` (largest first) until every replica is claimed.  With n_alone >= 0
  // (at most two replicas per SM) a block first prefers one replica: the first
  // block on an SM the next entry of `order` (`head`), the second block the
  // size-complement of its sibling's (entry n - 1 - (h - n_alone) for the
  // sibling's entry h), or none when the sibling's is among the n_alone largest.
  int* claimed;      // n_rep flags
  int* cursor;
  int* head;
  int* sm_slot;      // blocks seen per SM id (BHMC_SM_IDS entries)
  int* sm_head;      // entry + 1 taken by the first block of each SM id (0: not yet)
  int n_alone;       // -1: no pairing
};

#define BHMC_SM_IDS 1024

// --------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// --------------------------------------------------------------------------
// Exact depth-Dmax cell index: x * 2^Dmax / side is a power-of-two scaling
// (exact), floor is exact, so the cell equals the one reached by comparing x
// with every cluster mid-plane (ties to the upper half).
__device__ __forceinline__ unsigned long long spread3(unsigned long long v) {
  v &= 0x1fffffULL;
  v = (v | (v << 32)) & 0x1f00000000ffffULL;
  v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
  v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
  v = (v | (v << 2)) & 0x1249249249249249ULL;
  return v;
}

// Returns 0 if the point is outside the root cube (NaN and infinities included:
// the range test is done on the floored doubles before any integer conversion).
// Cell index floor(x * inv_hmin) - root_cell[a] along axis a, and whether it
// lies in [0, 2^Dmax).  inv_hmin = 2^s, so x * inv_hmin is exact and the floor
// can be read from the bits of x; tiny |x| (exponent below 2^-823, where the
// product could leave the normal range) takes the FP64 formula itself.
__device__ __forceinline__ bool cell_of(const SysDev& S, double x, int a, long long& c) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7ff);
  long long f;
  if (e == 0x7ff) return false;  // NaN or infinity
  if (e < 200) {
    const double ff = floor(__dmul_rn(x, S.inv_hmin)) - (double)S.root_cell[a];
    if (!(ff >= 0.0 && ff < (double)(1LL << S.Dmax))) return false;
    c = (long long)ff;
    return true;
  }
  const unsigned long long M = (u & 0xfffffffffffffULL) | (1ULL << 52);
  const int sh = e - 1075 + S.hmin_shift;  // |x| * 2^s = M * 2^sh
  if (sh >= 9) return false;                // |x| 2^s >= 2^61: outside the cube
  long long v;
  bool frac;
  if (sh >= 0) {
    v = (long long)(M << sh);
    frac = false;
  } else if (sh > -64) {
    v = (long long)(M >> -sh);
    frac = (M & ((1ULL << -sh) - 1ULL)) != 0ULL;
  } else {
    v = 0;
    frac = true;
  }
  f = (u >> 63) ? -v - (frac ? 1 : 0) : v;
  c = f - S.root_cell[a];
  return c >= 0 && c < (1LL << S.Dmax);
}

__device__ __forceinline__ unsigned long long point_key(const SysDev& S, double x, double y,
                                                        double z) {
  long long kx, ky, kz;
  if (!cell_of(S, x, 0, kx) || !cell_of(S, y, 1, ky) || !cell_of(S, z, 2, kz)) return 0ULL;
  return (1ULL << (3 * S.Dmax)) | spread3((unsigned long long)kx) | (spread3((unsigned long long)ky) << 1) |
         (spread3((unsigned long long)kz) << 2);
}

__device__ __forceinline__ int key_depth(unsigned long long k) { return (63 - __clzll(k)) / 3; }

// x = hi + lo with hi = round(x), lo = round(x - hi)
__device__ __forceinline__ float2 split2(double x) {
  float hi = __double2float_rn(x);
  float lo = __double2float_rn(__dsub_rn(x, (double)hi));
  return make_float2(hi, lo);
}

// Image of a charge q at r (FP64, same operation order as the definition:
// r2 = (x*x + y*y) + z*z, f = R*R / r2, image = f r, charge = ((alpha q) R) / |r|).
__device__ __forceinline__ bool image_of(const SysDev& S, const double r[3], double q,
                                         double out[3], double* qim) {
  double r2 = __dadd_rn(__dadd_rn(__dmul_rn(r[0], r[0]), __dmul_rn(r[1], r[1])),
                        __dmul_rn(r[2], r[2]));
  if (!(r2 > 0.0)) return false;
  double rn = __dsqrt_rn(r2);
  double f = __ddiv_rn(S.img_R2, r2);
  out[0] = __dmul_rn(f, r[0]);
  out[1] = __dmul_rn(f, r[1]);
  out[2] = __dmul_rn(f, r[2]);
  *qim = __ddiv_rn(__dmul_rn(__dmul_rn(S.img_alpha, q), S.img_R), rn);
  return true;
}

__device__ __forceinline__ bool in_root(const SysDev& S, const double x[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double hi = __dadd_rn(S.root_lo[a], S.root_side);
    if (!(x[a] >= S.root_lo[a]) || !(x[a] < hi)) return false;
  }
  return true;
}

__device__ __forceinline__ bool shell_ok(const SysDev& S, const double x[3]) {
  if (!S.shell) return true;
  double r2 = __dadd_rn(__dadd_rn(__dmul_rn(x[0], x[0]), __dmul_rn(x[1], x[1])),
                        __dmul_rn(x[2], x[2]));
  return r2 >= S.rmin2 && r2 <= S.rmax2;
}

// The running block's copy of its chain's error state (shared memory),
// raised together with the device error word so that a persistent kernel can
// test it between moves without a round trip to global memory.  A kernel that
// reads it first sets it from the error word.
__device__ __forceinline__ int& block_err() {
  __shared__ int e;
  return e;
}
__device__ __forceinline__ void set_err(const SysDev& S, int code) {
  atomicCAS(S.err, 0, code);
  block_err() = 1;
}

// Charge j is a fixed charge held outside the tree (fixed_direct).
__host__ __device__ __forceinline__ bool off_tree(const SysDev& S, int j) {
  return S.fixed_direct && j >= S.n_mob && j < S.n_mob + S.n_fix;
}

// Radial bin of a mobile ion at squared radius r2 (Sec. 4 RDF): r =
// sqrt(r2), k = floor((r - lo) / w) in FP64, -1 outside [lo, hi) or the bins.
__device__ __forceinline__ int rdf_bin(const SysDev& S, double r2) {
  const double r = __dsqrt_rn(r2);
  if (!(r >= S.rdf_lo && r < S.rdf_hi)) return -1;
  const double t = floor(__ddiv_rn(__dsub_rn(r, S.rdf_lo), S.rdf_w));
  return (t >= 0.0 && t < (double)S.rdf_nbins) ? (int)t : -1;
}

// Adds the running histogram to the accumulators `times` times (the samples
// of that many sample points taken in the same configuration); threads of
// the calling block share the bins.
__device__ __forceinline__ void rdf_sample(const SysDev& S, unsigned long long times) {
  if (!times) return;
  for (int k = threadIdx.x; k < S.rdf_nbins; k += blockDim.x) {
    S.rdf_acc[k] += times * S.rdf_run[k];
    S.rdf_accq[k] += (double)times * S.rdf_runq[k];
  }
  if (threadIdx.x == 0) *S.rdf_nsamp += times;
}

// Sample points among the moves [m0, m1): moves m with (m + 1) % every == 0.
__device__ __forceinline__ unsigned long long rdf_points(const SysDev& S, unsigned long long m0,
                                                         unsigned long long m1) {
  if (S.rdf_nbins <= 0 || S.rdf_every <= 0 || m1 <= m0) return 0ULL;
  const unsigned long long e = (unsigned long long)S.rdf_every;
  return m1 / e - m0 / e;
}

// Exact potential sum_f q_f / |r_f - x| at x of the fixed charges held outside
// the tree, in FP64 with the operation order of the definition; g (may be
// null) receives its gradient sum_f q_f (r_f - x) / |r_f - x|^3.
__device__ __forceinline__ double fixed_phi(const SysDev& S, const double x[3], double* g) {
  double phi = 0.0;
  if (g) g[0] = g[1] = g[2] = 0.0;
  for (int f = S.n_mob; f < S.n_mob + S.n_fix; ++f) {
    const double e[3] = {__dsub_rn(S.px[f], x[0]), __dsub_rn(S.py[f], x[1]), __dsub_rn(S.pz[f], x[2])};
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(e[0], e[0]), __dmul_rn(e[1], e[1])), __dmul_rn(e[2], e[2]));
    const double r = __dsqrt_rn(r2);
    const double qf = S.pq[f];
    phi = __dadd_rn(phi, __ddiv_rn(qf, r));
    if (g) {
      const double r3 = __dmul_rn(r2, r);
      for (int c = 0; c < 3; ++c) g[c] = __dadd_rn(g[c], __ddiv_rn(__dmul_rn(qf, e[c]), r3));
    }
  }
  return phi;
}

// Binomial coefficient C(n, m), 0 <= m <= n <= 10.
__device__ __forceinline__ int binom(int n, int m) {
  int c = 1;
  for (int k = 1; k <= m; ++k) c = c * (n - m + k) / k;
  return c;
}

// Moment term t (graded order) of charge q at offset d, in FP64 with the
// monomial built by repeated multiplication: q * ((dx^n1 * dy^n2) * dz^n3).
__device__ __forceinline__ void term_exponents(int t, int& n1, int& n2, int& n3) {
  int k = 0;
  while (nterms(k) <= t) ++k;
  int r = t - (k > 0 ? nterms(k - 1) : 0);
  int a = 0;  // a = k - n1: block of size a+1
  while ((a + 1) * (a + 2) / 2 <= r) ++a;
  int w = r - a * (a + 1) / 2;  // = a - n2
  n1 = k - a;
  n2 = a - w;
  n3 = k - n1 - n2;
}

__device__ __forceinline__ double mono_term(int n1, int n2, int n3, double q, double dx, double dy,
                                            double dz) {
  double px = 1.0, py = 1.0, pz = 1.0;
  for (int k = 0; k < n1; ++k) px = __dmul_rn(px, dx);
  for (int k = 0; k < n2; ++k) py = __dmul_rn(py, dy);
  for (int k = 0; k < n3; ++k) pz = __dmul_rn(pz, dz);
  return __dmul_rn(q, __dmul_rn(__dmul_rn(px, py), pz));
}

__device__ __forceinline__ int m32_index(const SysDev& S, int node, int t) {
  return S.layout == BHMC_LAYOUT_SOA ? t * S.node_cap + node : node * S.Kp + t;
}

// Evaluation coefficient W_t of a cluster from its FP64 moments (FP32 sums).
__device__ __forceinline__ void w_store(const SysDev& S, int node, int t) {
  const double* M = S.M64 + (size_t)node * S.K;
  float w = 0.f;
  for (int j = S.wrow[t]; j < S.wrow[t + 1]; ++j) w = fmaf(S.wval[j], __double2float_rn(M[S.wcol[j]]), w);
  S.W32[m32_index(S, node, t)] = w;
}

}  // namespace bhmc
