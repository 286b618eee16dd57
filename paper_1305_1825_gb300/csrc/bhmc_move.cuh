// bhmc_move.cuh -- one Metropolis trial move on the GPU: proposal (Philox),
// rejection tests, energy difference by the fused traversal at the old and new
// positions of the ion and its image (Sec. 1, Sec. 3.2), acceptance (Sec. 2)
// and the local adjustment of the octree (Sec. 3.3) with split/merge.
//
// A move is executed by one thread block (1, 2, 4 or 8 warps).  Serial control
// decisions are taken by thread 0; every loop over points, levels, moment
// terms or leaf slots is spread over the lanes.
#pragma once

#include "bhmc_block.cuh"

namespace bhmc {

// State of one trial move produced by its setup: the proposal, the four
// evaluation points and the rejection tests.
struct MoveSetup {
  TravPts T;
  int i, img, npts, nmov;
  double q, qa_img, qb_img;
  double a[3], b[3], ai[3], bi[3];
  int outcome, flagged;
  int rej_dom, rej_shell, rej_img;
  double dE, alpha;
  float la;    // log(alpha) in FP32, for the Metropolis decision's fast path
  // the move's exact terms, formed in the setup: weight x potential of the
  // off-tree fixed charges at every point, plus the ion-image pair terms
  double fix;
  int bin_a, bin_b;  // radial bins of the ion's old and new position (radial sampling on)
};

struct MoveSh : MoveSetup {
  int path[4][BHMC_MAX_D + 1];
  int pcnt[4][BHMC_MAX_D + 1];  // pre-move counts of the path clusters (BHMC_PCNT_LEAF: a leaf)
  int plen[4];
  int leafcnt[4];          // pre-move counts of the four path leaves
  int slot_i, slot_img;    // pre-move leaf slots of the ion and its image
  int merge_d[2];          // topmost level to merge on each old path
  int may_split0;          // a new leaf exceeds the split threshold when nothing merges
  int cnt[BHMC_MAX_WARPS][5];
  int go;
  int hc_hit;              // gradient traversal: hard-core overlap at point 1
  double xi[3];            // Langevin proposals: normal variates
  double U[2], gU[2][3];   // single-ion energy and gradient at the old / new position
  double tphi[2], tgrad[2][3];  // per-role potential and gradient of the last gradient traversal
  int split_node, split_g;
  unsigned char ex[nterms(BHMC_MAX_P)][3];  // exponents of every moment term
  float4 tA[BHMC_MAX_C + 2], tB[BHMC_MAX_C + 2];  // leaf slots of a merge
  // the next move's setup, computed while this move is decided, and its move
  // index (~0: none)
  MoveSetup nxt;
  unsigned long long nxt_m;
  int moved;  // ion moved by the last move (-1: none), which voids a setup of it
  double E;   // running FP64 energy of the chain while a kernel holds it
  // outcome and flag of the last finished move, for reads after its final
  // barrier: the next move's setup copy may already have overwritten the
  // MoveSetup fields by then, while these change only after every thread has
  // passed the next move's first barrier
  int result, result_flagged;
};

struct MoveStore {
  MoveSh sh;
  union {
    BlockStore bs;
    // (r - r_A)^k per moved charge, old/new position, level, axis
    double pw[2][2][BHMC_MAX_D + 1][3][BHMC_MAX_P + 1];
  };
};

// Per-kernel initialisation of the moment-term exponent table.
__device__ __forceinline__ void init_tables(MoveSh& sh, int K) {
  for (int t = threadIdx.x; t < K; t += blockDim.x) {
    int n1, n2, n3;
    term_exponents(t, n1, n2, n3);
    sh.ex[t][0] = (unsigned char)n1;
    sh.ex[t][1] = (unsigned char)n2;
    sh.ex[t][2] = (unsigned char)n3;
  }
}

// Role r of the setup runs on warp wb + r when the block has it, else on
// lanes 8r..8r+7 of warp wb; k is the lane within the role.
__device__ __forceinline__ bool setup_role(int r, int wb, int& k, int& base) {
  const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w = W > wb + r ? wb + r : wb;
  base = W > wb + r ? 0 : 8 * r;
  k = lane - base;
  return warp == w && k >= 0 && k < 8;
}

// Lanes base..base+2 hold coordinate k of a point x: the depth-Dmax key of x
// (0 outside the root cube, as point_key) in every lane, and
// r2 = (x0*x0 + x1*x1) + x2*x2 in every lane (FP64, the order of the definition).
__device__ __forceinline__ unsigned long long lane_key(const SysDev& S, double xk, int k, int base,
                                                       unsigned m3) {
  long long ck;
  const bool ok = cell_of(S, xk, k, ck);
  unsigned long long c = ok ? (spread3((unsigned long long)ck) << k) : 0ULL;
  const unsigned okm = __ballot_sync(m3, ok);
  c |= __shfl_sync(m3, c, base + 1) | __shfl_sync(m3, c, base + 2);
  c = __shfl_sync(m3, c, base);
  return ((okm >> base) & 7u) == 7u ? ((1ULL << (3 * S.Dmax)) | c) : 0ULL;
}
__device__ __forceinline__ double lane_r2(double xk, int base, unsigned m3) {
  const double sq = __dmul_rn(xk, xk);
  const double s1 = __shfl_sync(m3, sq, base + 1), s2 = __shfl_sync(m3, sq, base + 2);
  const double s0 = __shfl_sync(m3, sq, base);
  return __dadd_rn(__dadd_rn(s0, s1), s2);
}

// Proposal of move m (Sec. 2, uniform displacement): lanes 0-2 of warp wb
// form coordinate k of the trial position from Philox block (m, replica, 0),
// lane 3 forms alpha from block (m, replica, 1).
__device__ __forceinline__ void propose(const SysDev& S, MoveSetup& sh, unsigned long long m, unsigned replica,
                                        uint2 key, double step, int wb) {
  if ((int)(threadIdx.x >> 5) != wb || (threadIdx.x & 31) >= 4) return;
  const int k = threadIdx.x & 31;
  const uint4 u = philox(make_uint4((unsigned)m, (unsigned)(m >> 32), replica, k < 3 ? 0u : 1u), key);
  if (k < 3) {
    const int i = (int)(((unsigned long long)u.x * (unsigned long long)S.n_mob) >> 32);
    const unsigned uk = k == 0 ? u.y : (k == 1 ? u.z : u.w);
    const double src = (k == 0 ? S.px : (k == 1 ? S.py : S.pz))[i];
    // (u 2^-32 + 2^-33) - 1/2 = (2u + 1 - 2^32) 2^-33 exactly (every step of the
    // left side is exact in FP64), from one integer conversion
    const double unit = __ll2double_rn(2LL * (long long)uk + 1LL - (1LL << 32)) * 0x1p-33;
    sh.b[k] = __dadd_rn(src, __dmul_rn(unit, step));
    if (k == 0) {
      sh.i = i;
      sh.dE = 0.0;
      sh.flagged = 0;
    }
  } else {
    sh.alpha = __ll2double_rn(2LL * (long long)u.x + 1LL) * 0x1p-33;  // (u + 1/2) 2^-32 exactly
    sh.la = logf((float)sh.alpha);
  }
}

// Set up the move of ion sh.i to sh.b (all threads; sh.i and sh.b written
// before a barrier).  FP64 is slow on this part, so its work is spread over
// lanes (x, y, z side by side) and warps: role 0 the ion and the trial point's
// key and shell test, role 1 the trial image and its key, role 2 the image
// charge.  Sets sh.outcome = -1 to proceed or the rejection outcome, with the
// tests in the oracle's order: root cube, shell, image, image in root cube.
static __device__ void setup_roles(const SysDev& S, MoveSetup& sh, int wb) {
  TravPts& T = sh.T;
  const int i = sh.i;
  int k, base;
  // The lanes of a role first load one 8-byte value each in a single
  // instruction (divergent loads would wait for one another), then compute.
  if (setup_role(0, wb, k, base)) {
    const unsigned m3 = 7u << base;
    const unsigned long long* src =
        reinterpret_cast<const unsigned long long*>(k < 3 ? (k == 0 ? S.px : (k == 1 ? S.py : S.pz)) : S.pq);
    const unsigned long long val = k == 4 ? S.ckey[i] : src[i];  // a_k, q, key of the ion
    if (k < 3) {
      const double bk = sh.b[k];
      const unsigned long long kb = lane_key(S, bk, k, base, m3);
      const double r2 = lane_r2(bk, base, m3);
      if (S.rdf_nbins > 0) {  // radial bins of the old (lane 1) and new (lane 0) position
        const double r2a = lane_r2(__longlong_as_double((long long)val), base, m3);
        if (k == 0) sh.bin_b = rdf_bin(S, r2);
        if (k == 1) sh.bin_a = rdf_bin(S, r2a);
      }
      if (k == 0) {
        T.pkey[1] = kb;
        sh.rej_dom = kb == 0ULL;  // outside the root cube
        sh.rej_shell = S.shell ? !(r2 >= S.rmin2 && r2 <= S.rmax2) : 0;
        sh.npts = S.images ? 4 : 2;
        sh.nmov = S.images ? 2 : 1;
        T.n_excl = sh.nmov;
        T.excl[0] = i;
      }
      sh.a[k] = __longlong_as_double((long long)val);
    } else if (k == 3) {
      sh.q = __longlong_as_double((long long)val);
    } else if (k == 4) {
      T.pkey[0] = val;
      T.ekey[0] = val;
    }
  }
  if (setup_role(1, wb, k, base)) {
    const unsigned m3 = 7u << base;
    if (!S.images) {
      if (k == 0) {
        sh.rej_img = 0;
        sh.qa_img = 0.0;
      }
    } else {
      const int img = S.n_mob + S.n_fix + i;
      const unsigned long long* src =
          reinterpret_cast<const unsigned long long*>(k < 3 ? (k == 0 ? S.px : (k == 1 ? S.py : S.pz)) : S.pq);
      const unsigned long long val = k == 4 ? S.ckey[img] : src[img];  // a'_k, q', key of the image
      if (k < 3) {
        const double bk = sh.b[k];
        const double r2 = lane_r2(bk, base, m3);
        double bik = 0.0;
        unsigned long long kb = 0ULL;
        if (r2 > 0.0) {
          bik = __dmul_rn(__ddiv_rn(S.img_R2, r2), bk);
          kb = lane_key(S, bik, k, base, m3);
        }
        sh.bi[k] = kb ? bik : 0.0;
        sh.ai[k] = __longlong_as_double((long long)val);
        if (k == 0) {
          T.pkey[3] = kb;
          sh.rej_img = kb == 0ULL;
          sh.img = img;
          T.excl[1] = img;
        }
      } else if (k == 3) {
        sh.qa_img = __longlong_as_double((long long)val);
      } else if (k == 4) {
        T.pkey[2] = val;
        T.ekey[1] = val;
      }
    }
  }
  if (setup_role(2, wb, k, base)) {
    const unsigned m3 = 7u << base;
    if (!S.images) {
      if (k == 0) sh.qb_img = 0.0;
    } else if (k < 3) {
      const double r2 = lane_r2(sh.b[k], base, m3);
      if (k == 0) {
        double qb = 0.0;
        if (r2 > 0.0) qb = __ddiv_rn(__dmul_rn(__dmul_rn(S.img_alpha, S.pq[i]), S.img_R), __dsqrt_rn(r2));
        sh.qb_img = qb;
      }
    }
  }
}

// Outcome of the rejection tests, float pairs of the points and weights (warp
// wb).  Every lane converts one value in the same instruction stream: lane l <
// 12 coordinate l % 3 of point l / 3, 12-15 the weight of point l - 12, 16-17
// the charge of excluded charge l - 16.
static __device__ void setup_finish(const SysDev& S, MoveSetup& sh, int wb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp != wb) return;
  TravPts& T = sh.T;
  const int np = sh.npts;
  const int s = lane / 3, k = lane - 3 * (lane / 3);
  double v = 0.0;
  if (lane < 12) {
    const double* pts[4] = {sh.a, sh.b, sh.ai, sh.bi};
    if (s < np) v = pts[s][k];
  } else if (lane < 16) {
    const int t = lane - 12;
    v = t == 0 ? -sh.q : (t == 1 ? sh.q : (t == 2 ? -sh.qa_img : (sh.rej_img ? 0.0 : sh.qb_img)));
  } else if (lane < 18) {
    v = lane == 16 ? sh.q : sh.qa_img;
  }
  const float hi = __double2float_rn(v);
  const float lo = __double2float_rn(__dsub_rn(v, (double)hi));
  if (lane < 12) {
    if (s < np) {
      T.x[s][k] = v;
      T.hi[s][k] = hi;
      T.lo[s][k] = lo;
      reinterpret_cast<float*>(&T.h4[s])[k] = hi;
      reinterpret_cast<float*>(&T.l4[s])[k] = lo;
      if (s == 0 || s == 2) {
        T.ex[s >> 1][k] = v;
        T.ehi[s >> 1][k] = hi;
        T.elo[s >> 1][k] = lo;
      }
    } else {
      // unused points sit far outside the root so that they never touch a cluster
      reinterpret_cast<float*>(&T.h4[s])[k] = 3.0e38f;
      reinterpret_cast<float*>(&T.l4[s])[k] = 0.0f;
      if (k == 0) T.pkey[s] = 0ULL;
    }
  } else if (lane < 16) {
    const int t = lane - 12;
    if (t < np) {
      T.w64[t] = v;
      T.w[t] = hi;
    }
  } else if (lane < 18) {
    const int t = lane - 16;
    if (t < sh.nmov) {
      T.eq[t] = v;
      T.eqf[t] = hi;
    }
  } else if (lane == 31) {
    sh.outcome = sh.rej_dom ? BHMC_REJECT_DOMAIN
                            : sh.rej_shell ? BHMC_REJECT_OVERLAP : sh.rej_img ? BHMC_REJECT_DOMAIN : -1;
  }
  // fixed charges held outside the tree: their exact terms at every point
  // (FP64), one (point, fixed charge) pair per lane, summed over the warp
  // (1/r from one FP64 rsqrt, within an ulp: far below the FP64 parity bar)
  double fx = 0.0;
  if (S.fixed_direct) {
    const int s4 = lane & 3;
    if (s4 < np) {
      const double w = s4 == 0 ? -sh.q : (s4 == 1 ? sh.q : (s4 == 2 ? -sh.qa_img : (sh.rej_img ? 0.0 : sh.qb_img)));
      const double* x = s4 == 0 ? sh.a : (s4 == 1 ? sh.b : (s4 == 2 ? sh.ai : sh.bi));
      for (int f = S.n_mob + (lane >> 2); f < S.n_mob + S.n_fix; f += 8) {
        const double e0 = __dsub_rn(S.px[f], x[0]), e1 = __dsub_rn(S.py[f], x[1]), e2 = __dsub_rn(S.pz[f], x[2]);
        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(e0, e0), __dmul_rn(e1, e1)), __dmul_rn(e2, e2));
        fx = __dadd_rn(fx, __dmul_rn(__dmul_rn(w, S.pq[f]), rsqrt(r2)));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fx += __shfl_xor_sync(0xffffffffu, fx, o);
  }
  __syncwarp();
  if (lane == 0) {
    // ion-image pair terms q q'/|r - r'| at the new and old positions (in the
    // traversal's precision), formed here so that the move's decision waits
    // for none of this arithmetic
    double pair = 0.0;
    if (np == 4 && !(sh.rej_dom || sh.rej_shell || sh.rej_img)) {
      double pb, pa;
      if (S.prec == BHMC_PREC_F32) {
        float dx = (T.hi[1][0] - T.hi[3][0]) + (T.lo[1][0] - T.lo[3][0]);
        float dy = (T.hi[1][1] - T.hi[3][1]) + (T.lo[1][1] - T.lo[3][1]);
        float dz = (T.hi[1][2] - T.hi[3][2]) + (T.lo[1][2] - T.lo[3][2]);
        pb = (double)((float)(sh.q * sh.qb_img) * rsqrtf(dx * dx + dy * dy + dz * dz));
        dx = (T.hi[0][0] - T.hi[2][0]) + (T.lo[0][0] - T.lo[2][0]);
        dy = (T.hi[0][1] - T.hi[2][1]) + (T.lo[0][1] - T.lo[2][1]);
        dz = (T.hi[0][2] - T.hi[2][2]) + (T.lo[0][2] - T.lo[2][2]);
        pa = (double)((float)(sh.q * sh.qa_img) * rsqrtf(dx * dx + dy * dy + dz * dz));
      } else {
        double dx = sh.b[0] - sh.bi[0], dy = sh.b[1] - sh.bi[1], dz = sh.b[2] - sh.bi[2];
        pb = sh.q * sh.qb_img / sqrt(dx * dx + dy * dy + dz * dz);
        dx = sh.a[0] - sh.ai[0];
        dy = sh.a[1] - sh.ai[1];
        dz = sh.a[2] - sh.ai[2];
        pa = sh.q * sh.qa_img / sqrt(dx * dx + dy * dy + dz * dz);
      }
      pair = pb - pa;
    }
    sh.fix = fx + pair;
  }
}

static __device__ void setup_move(const SysDev& S, MoveSetup& sh) {
  setup_roles(S, sh, 0);
  __syncthreads();
  setup_finish(S, sh, 0);
}

// Paths and path leaf counts of a move not yet found (all threads).
__device__ __forceinline__ void clear_paths(MoveSh& sh) {
  for (int k = threadIdx.x; k < 4 * (BHMC_MAX_D + 1); k += blockDim.x) {
    (&sh.path[0][0])[k] = -1;
    (&sh.pcnt[0][0])[k] = BHMC_PCNT_NONE;
  }
  if (threadIdx.x < 4) sh.leafcnt[threadIdx.x] = -1;
}

// All warps: traverse, then thread 0 assembles dE (FP64).  Requires a
// __syncthreads() after setup (and after clear_paths when init_paths is
// false).  Returns with sh.dE and sh.cnt filled.
template <int P, typename Real, int LAYOUT>
__device__ void eval_move(const SysDev& S, MoveStore& st, bool record_path, bool init_paths = true) {
  MoveSh& sh = st.sh;
  if (init_paths) {
    clear_paths(sh);
    __syncthreads();
  }
  TravOut o;
  block_traverse<P, Real, LAYOUT>(S, sh.T, st.bs, sh.npts == 4 ? 15u : 3u, record_path ? sh.path : nullptr,
                                  sh.pcnt, sh.leafcnt, o);
  if (threadIdx.x == 0) {
    const double s = o.sum + sh.fix;  // the traversal's sum and the setup's exact terms
    sh.cnt[0][0] = o.visited;
    sh.cnt[0][1] = o.accepted;
    sh.cnt[0][2] = o.pairs;
    sh.cnt[0][3] = o.fp64;
    sh.cnt[0][4] = o.err;
    sh.dE = S.lB * s;
    if (o.overlap) {  // hard core (Eq. 2.1): rejected as before evaluation
      sh.outcome = BHMC_REJECT_OVERLAP;
      sh.dE = 0.0;
    }
  }
  __syncthreads();
}

// Complete the cluster paths of the points by descending from the deepest
// recorded cluster, and read the path leaves' counts (threads 0..npts-1).  A
// path the traversal followed down to its leaf needs no memory access.
static __device__ void complete_paths(const SysDev& S, MoveSh& sh) {
  const int s = threadIdx.x;
  if (s < sh.npts) {
    int d = 0;
    if (sh.path[s][0] < 0) sh.path[s][0] = 0;
    while (d < S.Dmax && sh.path[s][d + 1] >= 0) ++d;
    // the clusters' counts the traversal did not record (none, as a rule)
    for (int u = 0; u <= d; ++u)
      if (sh.pcnt[s][u] == BHMC_PCNT_NONE) {
        const int4 bu = S.nB[sh.path[s][u]];
        sh.pcnt[s][u] = bu.x >= 0 ? bu.y : BHMC_PCNT_LEAF;
      }
    if (sh.leafcnt[s] >= 0) {
      sh.plen[s] = d;
      return;
    }
    int node = sh.path[s][d];
    int4 b = S.nB[node];
    while (b.x >= 0 && d < S.Dmax) {
      const int o = (int)((sh.T.pkey[s] >> (3 * (S.Dmax - d - 1))) & 7ULL);
      node = b.x + o;
      ++d;
      sh.path[s][d] = node;
      b = S.nB[node];
      sh.pcnt[s][d] = b.x >= 0 ? b.y : BHMC_PCNT_LEAF;
    }
    sh.plen[s] = d;
    sh.leafcnt[s] = b.y;
  }
}

// Capacity rule (thread 0): after the move no depth-Dmax cell may hold more
// than C charges.  The common case is settled from the leaf counts alone.
static __device__ bool capacity_violation(const SysDev& S, const MoveSh& sh) {
  for (int s = 1; s < sh.npts; s += 2) {
    const int L = sh.path[s][sh.plen[s]];
    const int sh3 = 3 * (S.Dmax - sh.plen[s]);
    const unsigned long long kL = sh.T.pkey[s] >> sh3;
    int bound = sh.leafcnt[s];
    for (int u = 1; u < sh.npts; u += 2) bound += ((sh.T.pkey[u] >> sh3) == kL) ? 1 : 0;
    for (int u = 0; u < sh.T.n_excl; ++u) bound -= ((sh.T.ekey[u] >> sh3) == kL) ? 1 : 0;
    if (bound <= S.C) continue;  // the whole leaf stays within capacity
    const unsigned long long kb = sh.T.pkey[s];
    const int c = sh.leafcnt[s];
    int n = 0;
    for (int k = 0; k < c; ++k) {
      const int j = __float_as_int(S.sB[L * (S.C + 2) + k].w);
      bool ex = false;
      for (int u = 0; u < sh.T.n_excl; ++u) ex |= (sh.T.excl[u] == j);
      if (!ex && S.ckey[j] == kb) ++n;
    }
    for (int u = 1; u < sh.npts; u += 2) n += (sh.T.pkey[u] == kb) ? 1 : 0;
    if (n > S.C) return true;
  }
  return false;
}

__device__ __forceinline__ void mirror(const SysDev& S, int node, int t, double v) {
  if (S.prec == BHMC_PREC_F32) S.M32[m32_index(S, node, t)] = __double2float_rn(v);
}

__device__ __forceinline__ int* count_ptr(const SysDev& S, int node) {
  return reinterpret_cast<int*>(&S.nB[node]) + 1;
}
__device__ __forceinline__ int* child_ptr(const SysDev& S, int node) {
  return reinterpret_cast<int*>(&S.nB[node]);
}

static __device__ int alloc_group(const SysDev& S) {
  if (S.pool[1] > 0) return S.free_list[--S.pool[1]];
  if (S.pool[0] < S.group_cap) return S.pool[0]++;
  return -1;
}

static __device__ void free_group(const SysDev& S, int g) { S.free_list[S.pool[1]++] = g; }

// Merge (thread 0): cluster A becomes a leaf holding every particle of its subtree.
static __device__ void merge_cluster(const SysDev& S, MoveSh& sh, int A) {
  const int SC = S.C + 2;
  constexpr int kStack = 8 * 2 * (BHMC_MAX_D + 1) + 8;
  int stack[kStack];
  int top = 0, n = 0;
  const int g0 = S.nB[A].x;
  for (int o = 7; o >= 0; --o) stack[top++] = g0 + o;
  free_group(S, g0 >> 3);
  while (top > 0) {
    const int X = stack[--top];
    const int4 b = S.nB[X];
    if (b.x >= 0) {
      if (top + 8 > kStack) {  // cannot happen in a canonical tree
        set_err(S, BHMC_ESTACK);
        return;
      }
      for (int o = 7; o >= 0; --o) stack[top++] = b.x + o;
      free_group(S, b.x >> 3);
    } else {
      for (int k = 0; k < b.y && n < BHMC_MAX_C + 2; ++k) {
        sh.tA[n] = S.sA[X * SC + k];
        sh.tB[n] = S.sB[X * SC + k];
        ++n;
      }
    }
  }
  for (int k = 0; k < n; ++k) {
    S.sA[A * SC + k] = sh.tA[k];
    S.sB[A * SC + k] = sh.tB[k];
    const int j = __float_as_int(sh.tB[k].w);
    S.leaf_of[j] = A;
    S.slot_of[j] = k;
  }
  *child_ptr(S, A) = -1;
}

// Leaf slot operations of the moved charges (thread 0), from the pre-move leaf
// counts: delete = refill the slot with the leaf's last one, add = append.
static __device__ void move_slots(const SysDev& S, MoveSh& sh) {
  const int SC = S.C + 2;
  int LA[2], LB[2], cA[2], cB[2];
  for (int m = 0; m < sh.nmov; ++m) {
    LA[m] = sh.path[2 * m][sh.plen[2 * m]];
    LB[m] = sh.path[2 * m + 1][sh.plen[2 * m + 1]];
    cA[m] = sh.leafcnt[2 * m];
    cB[m] = sh.leafcnt[2 * m + 1];
  }
  if (sh.nmov > 1 && LA[0] != LB[0]) {  // leaf counts as the image sees them
    cA[1] += (LA[1] == LB[0]) - (LA[1] == LA[0]);
    cB[1] += (LB[1] == LB[0]) - (LB[1] == LA[0]);
  }
  int slot[2] = {sh.slot_i, sh.slot_img};
  for (int m = 0; m < sh.nmov; ++m) {
    const int j = m ? sh.img : sh.i;
    const double* B_ = m ? sh.bi : sh.b;
    const double qb = m ? sh.qb_img : sh.q;
    const int pb = 2 * m + 1;
    const float4 na4 = make_float4(sh.T.hi[pb][0], sh.T.hi[pb][1], sh.T.hi[pb][2], (float)qb);
    const float4 nb4 = make_float4(sh.T.lo[pb][0], sh.T.lo[pb][1], sh.T.lo[pb][2], __int_as_float(j));
    if (LA[m] == LB[m]) {
      S.sA[LA[m] * SC + slot[m]] = na4;
      S.sB[LA[m] * SC + slot[m]] = nb4;
    } else {
      const int k = slot[m], last = cA[m] - 1;
      if (k != last) {
        const float4 la = S.sA[LA[m] * SC + last], lb = S.sB[LA[m] * SC + last];
        S.sA[LA[m] * SC + k] = la;
        S.sB[LA[m] * SC + k] = lb;
        const int moved = __float_as_int(lb.w);
        S.slot_of[moved] = k;
        if (m == 0 && sh.nmov > 1 && moved == sh.img) slot[1] = k;
      }
      S.sA[LB[m] * SC + cB[m]] = na4;
      S.sB[LB[m] * SC + cB[m]] = nb4;
      S.leaf_of[j] = LB[m];
      S.slot_of[j] = cB[m];
    }
    S.px[j] = B_[0];
    S.py[j] = B_[1];
    S.pz[j] = B_[2];
    S.pq[j] = qb;
    S.ckey[j] = sh.T.pkey[pb];
  }
  if (S.rdf_nbins > 0) {  // the running radial histogram follows the moved ion
    if (sh.bin_a >= 0) {
      S.rdf_run[sh.bin_a] -= 1ULL;
      S.rdf_runq[sh.bin_a] -= sh.q;
    }
    if (sh.bin_b >= 0) {
      S.rdf_run[sh.bin_b] += 1ULL;
      S.rdf_runq[sh.bin_b] += sh.q;
    }
  }
}

// Barrier of the first n threads: the whole block (bar 0) or a named barrier.
// Named barriers use the non-aligned form (threads arrive one by one), which
// stays correct when a warp reaches it diverged after a lane-dependent branch;
// the aligned form requires a converged warp, and the compiler does not
// reconverge warps ahead of inline assembly.
__device__ __forceinline__ void team_sync(int bar, int n) {
  if (bar == 0)
    __syncthreads();
  else
    asm volatile("barrier.sync %0, %1;" ::"r"(bar), "r"(n) : "memory");
}

// (A0) of the local adjustment (Sec. 3.3): q (r - r_A)^k, (r - r_A)^k along
// the old and new paths of both moved charges in FP64, one thread per
// (charge, side, level, axis) with the powers built by repeated
// multiplication (the charge folded into the x powers), the merge and split
// tests, and the pre-move leaf slots.  Threads t0 .. t0 + n - 1 run it; it
// reads only the move's setup and its complete paths, so it may run before
// the Metropolis decision.
static __device__ void commit_prep(const SysDev& S, MoveStore& st, int t0, int n) {
  MoveSh& sh = st.sh;
  const int P = S.p;
  const int tid = (int)threadIdx.x - t0;
  if (tid < 0 || tid >= n) return;
  // one lane per (path, level, axis) of the moved charges' paths, packed on
  // consecutive lanes: each lane multiplies out one axis's powers (the
  // charge folded into the x powers), so a lane's FP64 chain is P + 1 long
  int tot = 0;
  for (int ps = 0; ps < 2 * sh.nmov; ++ps) tot += sh.plen[ps] + 1;
  for (int it = tid; it < 3 * tot; it += n) {
    const int ax = it % 3;
    int ps = 0, d = it / 3;
    while (d > sh.plen[ps]) {
      d -= sh.plen[ps] + 1;
      ++ps;
    }
    const int m = ps >> 1, side = ps & 1;
    const int node = sh.path[ps][d];
    const float4 c = S.nA[node];
    const double* X = m ? (side ? sh.bi : sh.ai) : (side ? sh.b : sh.a);
    const double q = m ? (side ? sh.qb_img : sh.qa_img) : sh.q;
    const double dx = __dsub_rn(X[ax], (double)(ax == 0 ? c.x : (ax == 1 ? c.y : c.z)));
    // the cluster's FP64 moments, which the update reads after the decision
    if (ax == 0) prefetch_range(S.M64 + (size_t)node * S.K, S.K * (int)sizeof(double));
    double* pw = st.pw[m][side][d][ax];
    double v = ax == 0 ? q : 1.0;
    pw[0] = v;
    for (int k = 1; k <= P; ++k) {
      v = __dmul_rn(v, dx);
      pw[k] = v;
    }
  }
  // the merge test of (C) from the pre-move counts: after the move an
  // internal cluster X at level d of an old path holds its count minus the
  // moved charges that leave it plus those that enter it, and the topmost one
  // at or below the split threshold merges.  One warp per moved charge, one
  // lane per level (the tree holds at most 32 levels).
  {
    const int nwq = n >> 5, wq = tid >> 5, d = tid & 31;
    for (int m = nwq - 1 - wq; m >= 0 && m < sh.nmov; m += nwq) {
      unsigned cand = 0xffffffffu;
      if (d <= sh.plen[2 * m] && sh.pcnt[2 * m][d] != BHMC_PCNT_LEAF) {
        const int X = sh.path[2 * m][d];
        int c = sh.pcnt[2 * m][d];
        for (int u = 0; u < sh.nmov; ++u) {
          const int na = d <= sh.plen[2 * u] ? sh.path[2 * u][d] : -1;
          const int nb = d <= sh.plen[2 * u + 1] ? sh.path[2 * u + 1][d] : -1;
          if (na != nb) c += (nb == X) - (na == X);
        }
        if (c <= S.Cs) cand = (unsigned)d;
      }
      const unsigned dm = __reduce_min_sync(0xffffffffu, cand);
      if (d == 0) sh.merge_d[m] = dm == 0xffffffffu ? (1 << 20) : (int)dm;
    }
  }
  // the split test of (D) when nothing merges: the new leaves' counts follow
  // from their pre-move counts
  if (tid == n - 3) {
    int ms = 0;
    for (int m = 0; m < sh.nmov; ++m) {
      const int L = sh.path[2 * m + 1][sh.plen[2 * m + 1]];
      int c = sh.leafcnt[2 * m + 1];
      for (int u = 0; u < sh.nmov; ++u) {
        const int ua = sh.path[2 * u][sh.plen[2 * u]], ub = sh.path[2 * u + 1][sh.plen[2 * u + 1]];
        if (ua != ub) c += (ub == L) - (ua == L);
      }
      if (c > S.Cs) ms = 1;
    }
    sh.may_split0 = ms;
  }
  if (tid == n - 1) sh.slot_i = S.slot_of[sh.i];
  if (tid == n - 2 && sh.nmov > 1) sh.slot_img = S.slot_of[sh.img];
}

// Index of the first of the four path clusters (old/new of the ion, old/new
// of the image) that holds the same cluster as a[k] (k itself when none before it does).
__device__ __forceinline__ int first_of(const int a[4], int k) {
  for (int j = 0; j < k; ++j)
    if (a[j] == a[k]) return j;
  return k;
}

// v[k] and v[k] = x for a run-time k in 0..3 without indexing the array
// (selects keep it in registers).
__device__ __forceinline__ double pick4(const double v[4], int k) {
  return k == 0 ? v[0] : k == 1 ? v[1] : k == 2 ? v[2] : v[3];
}
__device__ __forceinline__ void put4(double v[4], int k, double x) {
  v[0] = k == 0 ? x : v[0];
  v[1] = k == 1 ? x : v[1];
  v[2] = k == 2 ? x : v[2];
  v[3] = k == 3 ? x : v[3];
}

// Local adjustment (Sec. 3.3) of an accepted move after commit_prep.  The
// first nt threads of the block (all when nt == 0) run it, synchronised by
// barrier `bar` (0: __syncthreads).
static __device__ void commit_apply(const SysDev& S, MoveStore& st, int nt, int bar) {
  MoveSh& sh = st.sh;
  const int K = S.K, SC = S.C + 2;
  const int tid = threadIdx.x, nth = nt > 0 ? nt : (int)blockDim.x;
  constexpr int NL = BHMC_MAX_D + 1;
  // (A1) FP64 moments per level, both moved charges in one pass: one thread
  // owns each (level, term), the four path clusters of that level (a cluster
  // belongs to one level) are read together, then the ion's update and the
  // image's are applied in that order (M_old -= ma, M_new += mb; one cluster
  // may be both) and each distinct cluster written once.  Each update is one
  // FP64 fused multiply-add of q x^n1 y^n2 by z^n3.  The last thread moves
  // the leaf slots meanwhile.
  {
    int Dn = 0;
    for (int ps = 0; ps < 2 * sh.nmov; ++ps) Dn = max(Dn, sh.plen[ps] + 1);
    const int nw = nth - 1;
    if (tid == nw) move_slots(S, sh);
    for (int it = tid; tid < nw && it < Dn * K; it += nw) {
      const int d = it / K, t = it - d * K;
      const int n1 = sh.ex[t][0], n2 = sh.ex[t][1], n3 = sh.ex[t][2];
      int a[4];
      double v[4], pxy[4], pz[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) a[k] = (k < 2 * sh.nmov && d <= sh.plen[k]) ? sh.path[k][d] : -1;
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = a[k] >= 0 ? S.M64[(size_t)a[k] * K + t] : 0.0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int m = k >> 1, side = k & 1;
        const bool on = a[k] >= 0;
        pxy[k] = on ? __dmul_rn(st.pw[m][side][d][0][n1], st.pw[m][side][d][1][n2]) : 0.0;
        pz[k] = on ? st.pw[m][side][d][2][n3] : 0.0;
      }
      int own[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) own[k] = first_of(a, k);
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        const int ka = 2 * m, kb = 2 * m + 1;
        const bool same = a[ka] >= 0 && a[ka] == a[kb];
        if (a[ka] >= 0) {  // old cluster: M -= ma, then M += mb when it is also the new one
          double x = __fma_rn(-pxy[ka], pz[ka], pick4(v, own[ka]));
          if (same) x = __fma_rn(pxy[kb], pz[kb], x);
          put4(v, own[ka], x);
        }
        if (a[kb] >= 0 && !same) put4(v, own[kb], __fma_rn(pxy[kb], pz[kb], pick4(v, own[kb])));
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (a[k] >= 0 && own[k] == k) {
          S.M64[(size_t)a[k] * K + t] = v[k];
          mirror(S, a[k], t, v[k]);
        }
    }
    for (int it = tid; it < sh.nmov * NL; it += nth) {
      const int mm = it / NL, d = it - mm * NL;
      const int pa2 = 2 * mm, pb2 = 2 * mm + 1;
      const int na = d <= sh.plen[pa2] ? sh.path[pa2][d] : -1;
      const int nb = d <= sh.plen[pb2] ? sh.path[pb2][d] : -1;
      if (na != nb) {
        if (na >= 0) atomicSub(count_ptr(S, na), 1);
        if (nb >= 0) atomicAdd(count_ptr(S, nb), 1);
      }
    }
  }
  // commit_prep found what merges (merge_d) and whether a new leaf may split
  // when nothing merges (may_split0); in the common case neither happens and
  // the caller's block barrier ends the commit
  const bool merge = sh.merge_d[0] < NL || (sh.nmov > 1 && sh.merge_d[1] < NL);
  const bool may_split = merge || sh.may_split0 != 0;
  if (!may_split) return;
  team_sync(bar, nth);
  // (C) merge the topmost internal cluster on an old path holding no more
  // charges than the split threshold after the move
  if (merge) {
    if (tid == 0) {
      const int d0 = sh.merge_d[0];
      if (d0 < NL) merge_cluster(S, sh, sh.path[0][d0]);
      if (sh.nmov > 1) {
        const int d1 = sh.merge_d[1];
        const bool inside = d0 < NL && d1 >= d0 && sh.path[2][d0] == sh.path[0][d0];
        if (d1 < NL && !inside) merge_cluster(S, sh, sh.path[2][d1]);
      }
    }
    team_sync(bar, nth);
  }
  // (D) split the new leaves while they hold more charges than the split threshold
  for (int m = 0; m < sh.nmov; ++m) {
    const int j = m ? sh.img : sh.i;
    for (int guard = 0; guard <= BHMC_MAX_D; ++guard) {
      if (tid == 0) {
        const int L = S.leaf_of[j];
        const int4 b = S.nB[L];
        const unsigned long long key = ((unsigned long long)(unsigned)b.w << 32) | (unsigned)b.z;
        const int dL = key_depth(key);
        sh.split_node = -1;
        if (b.y > S.Cs && dL < S.Dmax) {
          const int g = alloc_group(S);
          if (g < 0) {
            set_err(S, BHMC_ENOMEM_POOL);
          } else {
            const int c0 = 8 * g;
            const float4 a = S.nA[L];
            const float hc = 0.5f * a.w;
            for (int o = 0; o < 8; ++o) {
              const unsigned long long ck = (key << 3) | (unsigned long long)o;
              S.nA[c0 + o] = make_float4((o & 1) ? a.x + hc : a.x - hc, (o & 2) ? a.y + hc : a.y - hc,
                                         (o & 4) ? a.z + hc : a.z - hc, hc);
              S.nB[c0 + o] = make_int4(-1, 0, (int)(unsigned)(ck & 0xffffffffULL), (int)(unsigned)(ck >> 32));
            }
            const int sh3 = 3 * (S.Dmax - dL - 1);
            for (int k = 0; k < b.y; ++k) {
              const float4 ea = S.sA[L * SC + k], eb = S.sB[L * SC + k];
              const int idx = __float_as_int(eb.w);
              const int o = (int)((S.ckey[idx] >> sh3) & 7ULL);
              const int ch = c0 + o;
              const int pos = S.nB[ch].y;
              S.sA[ch * SC + pos] = ea;
              S.sB[ch * SC + pos] = eb;
              *count_ptr(S, ch) = pos + 1;
              S.leaf_of[idx] = ch;
              S.slot_of[idx] = pos;
            }
            *child_ptr(S, L) = c0;
            sh.split_node = L;
            sh.split_g = c0;
          }
        }
      }
      team_sync(bar, nth);
      if (sh.split_node < 0) break;
      for (int it = tid; it < 8 * K; it += nth) {
        const int o = it / K, t = it - o * K;
        const int ch = sh.split_g + o;
        const float4 c = S.nA[ch];
        const int cnt = S.nB[ch].y;
        const int n1 = sh.ex[t][0], n2 = sh.ex[t][1], n3 = sh.ex[t][2];
        double M = 0.0;
        for (int k = 0; k < cnt; ++k) {
          const int idx = __float_as_int(S.sB[ch * SC + k].w);
          M = __dadd_rn(M, mono_term(n1, n2, n3, S.pq[idx], __dsub_rn(S.px[idx], (double)c.x),
                                     __dsub_rn(S.py[idx], (double)c.y), __dsub_rn(S.pz[idx], (double)c.z)));
        }
        S.M64[(size_t)ch * K + t] = M;
        mirror(S, ch, t, M);
      }
      team_sync(bar, nth);
    }
  }
}

// Local adjustment (Sec. 3.3) of an accepted move.  Requires complete paths
// and leaf counts (complete_paths).  The first nt threads of the block (all
// when nt == 0) run it, synchronised by barrier `bar` (0: __syncthreads).
static __device__ void commit_move_block(const SysDev& S, MoveStore& st, int nt = 0, int bar = 0) {
  const int nth = nt > 0 ? nt : (int)blockDim.x;
  commit_prep(S, st, 0, nth);
  team_sync(bar, nth);
  commit_apply(S, st, nt, bar);
}

// ---------------------------------------------------------------------------
// Metropolis decision in FP64 (alpha <= exp(-beta dE)), settled in FP32 when
// the two sides differ by more than a safe margin.
__device__ __forceinline__ void metropolis(double beta, double dE, double alpha, float la, int& accept,
                                           int& flagged) {
  const double x = -beta * dE;
  const float xf = (float)x;
  const float diff = xf - la;
  const float margin = 1e-4f * (1.0f + fabsf(xf) + fabsf(la));
  if (diff > margin) {
    accept = 1;
    flagged = 0;
  } else if (diff < -margin) {
    accept = 0;
    flagged = 0;
  } else {
    accept = alpha <= exp(x) ? 1 : 0;
    flagged = fabs(x - log(alpha)) < 1e-6 ? 1 : 0;
  }
}

struct MoveRec {
  long long i;
  double r[3];
  double dE;
  int outcome, flagged;
};

// Barrier of warps 5-7 (the lookahead setup of the next move), non-aligned
// like team_sync's.
__device__ __forceinline__ void bar_ahead() { asm volatile("barrier.sync 1, 96;" ::: "memory"); }

// One full trial move m of a chain (all threads).  Returns the outcome, or -1
// after a device error (recorded in S.err).  With `ahead` (blocks of eight
// warps), warps 5-7 set up move m + 1 into sh.nxt while warps 0-4 decide and
// commit move m; move m + 1 uses it unless move m moved the same ion (the
// setup reads nothing else that a move changes), so the chain is unchanged.
template <int P, typename Real, int LAYOUT>
__device__ int mc_move(const SysDev& S, MoveStore& st, unsigned long long m, unsigned replica,
                       uint2 key, double step, MoveRec* rec, bool ahead) {
  MoveSh& sh = st.sh;
  const int warp = threadIdx.x >> 5;
  ahead = ahead && blockDim.x == 256;
  clear_paths(sh);  // nothing reads the paths before the barrier that ends the setup
  // the look-ahead setup of move m is used unless move m - 1 moved its ion
  // (both read after the barrier that ended move m - 1, so every thread agrees)
  if (sh.nxt_m == m && sh.nxt.i != sh.moved) {
    constexpr int n = (int)(sizeof(MoveSetup) / sizeof(int));
    int* dst = reinterpret_cast<int*>(static_cast<MoveSetup*>(&sh));
    const int* src = reinterpret_cast<const int*>(&sh.nxt);
    for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
  } else {
    propose(S, sh, m, replica, key, step, 0);
    __syncthreads();
    setup_roles(S, sh, 0);
    __syncthreads();
    setup_finish(S, sh, 0);
  }
  __syncthreads();
  if (threadIdx.x == 0) sh.nxt_m = ~0ULL;
  if (sh.outcome < 0) {
    eval_move<P, Real, LAYOUT>(S, st, true, false);
    if (sh.cnt[0][4]) {
      if (threadIdx.x == 0) set_err(S, sh.cnt[0][4]);
      return -1;
    }
    if (ahead && warp >= 5) {
      // warps 5-7: the next move's setup, while warps 0-4 decide and commit
      propose(S, sh.nxt, m + 1, replica, key, step, 5);
      bar_ahead();
      setup_roles(S, sh.nxt, 5);
      bar_ahead();
      setup_finish(S, sh.nxt, 5);
      if (threadIdx.x == 160) sh.nxt_m = m + 1;
    } else {
      const int nt = ahead ? 160 : (int)blockDim.x, bar = ahead ? 2 : 0;
      // warp 0 decides while the other warps of the team prepare the commit
      const bool early = nt > 32;
      complete_paths(S, sh);
      team_sync(bar, nt);
      if (threadIdx.x == 0 && sh.outcome < 0) {
        int acc, fl;
        metropolis(S.beta, sh.dE, sh.alpha, sh.la, acc, fl);
        sh.flagged = fl;
        if (!isfinite(sh.dE)) {
          set_err(S, BHMC_ENONFINITE);
          sh.outcome = BHMC_REJECT_ENERGY;
        } else if (!acc)
          sh.outcome = BHMC_REJECT_ENERGY;
        else if (capacity_violation(S, sh))
          sh.outcome = BHMC_REJECT_CAPACITY;
        else
          sh.outcome = BHMC_ACCEPT;
      }
      if (early) commit_prep(S, st, 32, nt - 32);
      team_sync(bar, nt);
      if (sh.outcome == BHMC_ACCEPT) {
        if (!early) {
          commit_prep(S, st, 0, nt);
          team_sync(bar, nt);
        }
        commit_apply(S, st, nt, bar);
        if (threadIdx.x == 0) sh.E += sh.dE;
      }
    }
  }
  if (threadIdx.x == 0) {
    // not a write of nxt_m here: thread 160 may still be finishing the
    // look-ahead, and its nxt_m = m + 1 must not undo an invalidation
    sh.moved = sh.outcome == BHMC_ACCEPT ? sh.i : -1;
    sh.result = sh.outcome;
    sh.result_flagged = sh.flagged;
    if (rec) {
      rec->i = sh.i;
      rec->r[0] = sh.b[0];
      rec->r[1] = sh.b[1];
      rec->r[2] = sh.b[2];
      rec->dE = sh.dE;
      rec->outcome = sh.outcome;
      rec->flagged = sh.flagged;
    }
  }
  __syncthreads();
  return sh.result;
}

// ---------------------------------------------------------------------------
// Metropolis-adjusted Langevin single-ion moves.  The single-ion energy is
//   U(x) = l_B [q phi(x) + q'(x) phi(x'(x)) + q q'(x) / |x - x'(x)|]
// on the pre-move tree with the ion and its image excluded (so that
// dE = U(b) - U(a) is the trial move's energy difference), with
// x' = R^2 x/|x|^2, q' = alpha q R/|x|:
//   grad U = l_B [q grad phi(x) + q' J^T grad phi(x') + phi(x') grad q' + grad P],
//   J = (R^2/|x|^2)(I - 2 x x^T/|x|^2), grad q' = -q' x/|x|^2,
//   P = alpha q^2 R / (|x|^2 - R^2), grad P = -2 alpha q^2 R x / (|x|^2 - R^2)^2.

// One gradient traversal over the points of pmask; results in sh.tphi, sh.tgrad.
template <int P, typename Real, int LAYOUT>
__device__ bool eval_grad(const SysDev& S, MoveStore& st, unsigned pmask) {
  MoveSh& sh = st.sh;
  for (int k = threadIdx.x; k < 4 * (BHMC_MAX_D + 1); k += blockDim.x)
    if ((pmask >> (k / (BHMC_MAX_D + 1))) & 1u) {
      (&sh.path[0][0])[k] = -1;
      (&sh.pcnt[0][0])[k] = BHMC_PCNT_NONE;
    }
  if (threadIdx.x < 4 && ((pmask >> threadIdx.x) & 1u)) sh.leafcnt[threadIdx.x] = -1;
  __syncthreads();
  TravOut o;
  block_traverse<P, Real, LAYOUT, true>(S, sh.T, st.bs, pmask, sh.path, sh.pcnt, sh.leafcnt, o);
  if (threadIdx.x == 0) {
    for (int r = 0; r < 2; ++r) {
      sh.tphi[r] = o.phi[r];
      for (int c = 0; c < 3; ++c) sh.tgrad[r][c] = o.grad[r][c];
    }
    if (S.fixed_direct) {
      // the off-tree fixed charges' exact potential and gradient at the point
      // of each role (role 0: point 0 or 1, role 1: point 2 or 3)
      for (int r = 0; r < 2; ++r) {
        const int s = 2 * r + (((pmask >> (2 * r)) & 1u) ? 0 : 1);
        if (!((pmask >> s) & 1u)) continue;
        double g[3];
        sh.tphi[r] += fixed_phi(S, sh.T.x[s], g);
        for (int c = 0; c < 3; ++c) sh.tgrad[r][c] += g[c];
      }
    }
    sh.cnt[0][4] = o.err;
    sh.hc_hit = o.overlap;
  }
  __syncthreads();
  return sh.cnt[0][4] == 0;
}

// U and grad U at x (image xi, image charge qimg) from a gradient traversal (thread 0).
__device__ __forceinline__ void ion_energy(const SysDev& S, const MoveSh& sh, const double x[3], const double xi[3],
                                           double qimg, double& U, double g[3]) {
  const double q = sh.q;
  double u = q * sh.tphi[0];
  for (int c = 0; c < 3; ++c) g[c] = q * sh.tgrad[0][c];
  if (S.images) {
    const double* g2 = sh.tgrad[1];
    const double R = S.img_R;
    const double r2 = (x[0] * x[0] + x[1] * x[1]) + x[2] * x[2];
    u += qimg * sh.tphi[1];
    const double dx = x[0] - xi[0], dy = x[1] - xi[1], dz = x[2] - xi[2];
    u += q * qimg / sqrt((dx * dx + dy * dy) + dz * dz);
    const double f = R * R / r2;
    const double xg = (x[0] * g2[0] + x[1] * g2[1]) + x[2] * g2[2];
    const double pden = r2 - R * R;
    for (int c = 0; c < 3; ++c) {
      g[c] += qimg * (f * (g2[c] - 2.0 * x[c] * xg / r2)) - sh.tphi[1] * qimg * x[c] / r2;
      g[c] += -S.img_alpha * q * q * R * 2.0 * x[c] / (pden * pden);
    }
  }
  U = S.lB * u;
  for (int c = 0; c < 3; ++c) g[c] *= S.lB;
}

template <int P, typename Real, int LAYOUT>
__device__ int mala_move(const SysDev& S, MoveStore& st, unsigned long long m, unsigned replica, uint2 key,
                         double tau, MoveRec* rec) {
  MoveSh& sh = st.sh;
  if (threadIdx.x == 0) {
    const uint4 u = philox(make_uint4((unsigned)m, (unsigned)(m >> 32), replica, 0u), key);
    const uint4 v = philox(make_uint4((unsigned)m, (unsigned)(m >> 32), replica, 1u), key);
    const uint4 w = philox(make_uint4((unsigned)m, (unsigned)(m >> 32), replica, 2u), key);
    const int i = (int)(((unsigned long long)u.x * (unsigned long long)S.n_mob) >> 32);
    const double un0 = ((double)w.x + 0.5) * 0x1p-32, un1 = ((double)w.y + 0.5) * 0x1p-32;
    const double un2 = ((double)w.z + 0.5) * 0x1p-32, un3 = ((double)w.w + 0.5) * 0x1p-32;
    const double two_pi = 6.283185307179586;
    const double rad0 = sqrt(-2.0 * log(un0)), rad1 = sqrt(-2.0 * log(un2));
    sh.xi[0] = rad0 * cos(two_pi * un1);
    sh.xi[1] = rad0 * sin(two_pi * un1);
    sh.xi[2] = rad1 * cos(two_pi * un3);
    sh.alpha = ((double)v.x + 0.5) * 0x1p-32;
    sh.i = i;
    sh.b[0] = S.px[i];
    sh.b[1] = S.py[i];
    sh.b[2] = S.pz[i];
    sh.dE = 0.0;
    sh.flagged = 0;
  }
  __syncthreads();
  setup_move(S, sh);  // points at the current position (b = a) for the first traversal
  __syncthreads();
  if (!eval_grad<P, Real, LAYOUT>(S, st, sh.npts == 4 ? 5u : 1u)) {
    if (threadIdx.x == 0) set_err(S, sh.cnt[0][4]);
    return -1;
  }
  if (threadIdx.x == 0) {
    ion_energy(S, sh, sh.a, sh.ai, sh.qa_img, sh.U[0], sh.gU[0]);
    const double tb = tau * S.beta, sd = sqrt(2.0 * tau);
    for (int c = 0; c < 3; ++c)
      sh.b[c] = __dadd_rn(__dsub_rn(sh.a[c], __dmul_rn(tb, sh.gU[0][c])), __dmul_rn(sd, sh.xi[c]));
  }
  __syncthreads();
  setup_move(S, sh);
  __syncthreads();
  if (sh.outcome < 0) {
    if (!eval_grad<P, Real, LAYOUT>(S, st, sh.npts == 4 ? 10u : 2u)) {
      if (threadIdx.x == 0) set_err(S, sh.cnt[0][4]);
      return -1;
    }
    complete_paths(S, sh);
    __syncthreads();
    if (threadIdx.x == 0 && sh.hc_hit) {  // hard core (Eq. 2.1) at the trial position
      sh.outcome = BHMC_REJECT_OVERLAP;
      sh.dE = 0.0;
    } else if (threadIdx.x == 0) {
      ion_energy(S, sh, sh.b, sh.bi, sh.qb_img, sh.U[1], sh.gU[1]);
      sh.dE = sh.U[1] - sh.U[0];
      const double tb = tau * S.beta;
      double fwd = 0.0, rev = 0.0;
      for (int c = 0; c < 3; ++c) {
        const double f = sh.b[c] - sh.a[c] + tb * sh.gU[0][c];
        const double g = sh.a[c] - sh.b[c] + tb * sh.gU[1][c];
        fwd += f * f;
        rev += g * g;
      }
      const double lacc = -S.beta * sh.dE - rev / (4.0 * tau) + fwd / (4.0 * tau);
      const double la = log(sh.alpha);
      sh.flagged = fabs(lacc - la) < 1e-6 ? 1 : 0;
      if (!(la <= lacc))
        sh.outcome = BHMC_REJECT_ENERGY;
      else if (capacity_violation(S, sh))
        sh.outcome = BHMC_REJECT_CAPACITY;
      else
        sh.outcome = BHMC_ACCEPT;
    }
    __syncthreads();
    if (sh.outcome == BHMC_ACCEPT) {
      commit_move_block(S, st);
      if (threadIdx.x == 0) *S.energy += sh.dE;
    }
  }
  if (threadIdx.x == 0 && rec) {
    rec->i = sh.i;
    rec->r[0] = sh.b[0];
    rec->r[1] = sh.b[1];
    rec->r[2] = sh.b[2];
    rec->dE = sh.dE;
    rec->outcome = sh.outcome;
    rec->flagged = sh.flagged;
  }
  __syncthreads();
  return sh.outcome;
}

__device__ __forceinline__ void tally(bhmc_mc_stats* st, int outcome, int flagged) {
  st->moves += 1;
  if (outcome == BHMC_ACCEPT) st->accepted += 1;
  if (outcome == BHMC_REJECT_ENERGY) st->rej_energy += 1;
  if (outcome == BHMC_REJECT_DOMAIN) st->rej_domain += 1;
  if (outcome == BHMC_REJECT_OVERLAP) st->rej_overlap += 1;
  if (outcome == BHMC_REJECT_CAPACITY) st->rej_capacity += 1;
  st->flagged += flagged;
}

// ---------------------------------------------------------------------------
// Kernels
struct DeltaOut {
  double dE;
  long long cnt[4];
  int status;
  int err;
};

template <int P, typename Real, int LAYOUT>
__global__ void __launch_bounds__(32 * BHMC_MAX_WARPS) k_delta(SysDev S, int i, double bx, double by, double bz,
                                               DeltaOut* out) {
  __shared__ MoveStore st;
  if (threadIdx.x == 0) {
    st.sh.i = i;
    st.sh.b[0] = bx;
    st.sh.b[1] = by;
    st.sh.b[2] = bz;
  }
  __syncthreads();
  setup_move(S, st.sh);
  __syncthreads();
  if (threadIdx.x == 0) {
    const int o = st.sh.outcome;
    out->status = o < 0 ? 0 : (o == BHMC_REJECT_DOMAIN ? BHMC_EDOMAIN : BHMC_EOVERLAP);
  }
  if (st.sh.outcome >= 0) return;
  eval_move<P, Real, LAYOUT>(S, st, false);
  if (threadIdx.x == 0) {
    const bool hit = st.sh.outcome >= 0;  // hard-core overlap at the trial point
    out->status = hit ? BHMC_EOVERLAP : 0;
    out->dE = st.sh.dE;
    for (int k = 0; k < 4; ++k) out->cnt[k] = hit ? 0 : st.sh.cnt[0][k];
    out->err = st.sh.cnt[0][4];
  }
}

template <int P, typename Real, int LAYOUT>
__global__ void __launch_bounds__(32 * BHMC_MAX_WARPS) k_step(SysDev S, unsigned long long m, unsigned replica,
                                              uint2 key, double step, MoveRec* recs,
                                              bhmc_mc_stats* stats) {
  __shared__ MoveStore st;
  if (*(volatile int*)S.err) return;
  init_tables(st.sh, S.K);
  if (threadIdx.x == 0) {
    st.sh.nxt_m = ~0ULL;
    st.sh.E = *S.energy;
  }
  __syncthreads();
  const int o = mc_move<P, Real, LAYOUT>(S, st, m, replica, key, step, recs, false);
  if (threadIdx.x == 0) *S.energy = st.sh.E;
  if (threadIdx.x == 0 && o >= 0) {
    tally(stats, o, st.sh.result_flagged);
    stats->energy = st.sh.E;
  }
  if (o >= 0) rdf_sample(S, rdf_points(S, m, m + 1));
}

template <int P, typename Real, int LAYOUT>
__global__ void __launch_bounds__(32 * BHMC_MAX_WARPS) k_step_mala(SysDev S, unsigned long long m, unsigned replica, uint2 key,
                                                   double tau, MoveRec* recs, bhmc_mc_stats* stats) {
  __shared__ MoveStore st;
  if (*(volatile int*)S.err) return;
  init_tables(st.sh, S.K);
  const int o = mala_move<P, Real, LAYOUT>(S, st, m, replica, key, tau, recs);
  if (threadIdx.x == 0 && o >= 0) {
    tally(stats, o, st.sh.flagged);
    stats->energy = *S.energy;
  }
  if (o >= 0) rdf_sample(S, rdf_points(S, m, m + 1));
}


__device__ __forceinline__ unsigned sm_id() {
  unsigned r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}

// The replica this block prefers for its first chain (thread 0), n_rep for
// none (see BatchArgs).  The second block on an SM waits for its sibling's
// choice, which the sibling publishes right after taking it (both are
// resident); the wait is bounded, and a block that gives up takes replicas
// from the cursor like any other.
__device__ __forceinline__ int batch_preferred(const BatchArgs* args, int n_rep) {
  const unsigned id = sm_id();
  if (id >= BHMC_SM_IDS) return n_rep;
  const int slot = atomicAdd(&args->sm_slot[id], 1);
  if (slot == 0) {
    const int h = atomicAdd(args->head, 1);
    atomicExch(&args->sm_head[id], h + 1);
    return h < n_rep ? args->order[h] : n_rep;
  }
  if (slot != 1) return n_rep;
  int v = 0;
  for (int it = 0; it < (1 << 16); ++it) {
    v = atomicAdd(&args->sm_head[id], 0);
    if (v) break;
    __nanosleep(256);
  }
  if (!v) return n_rep;
  const int h = v - 1;
  const int e = n_rep - 1 - (h - args->n_alone);
  return (h >= args->n_alone && e >= 0 && e < n_rep) ? args->order[e] : n_rep;
}

template <int P, typename Real, int LAYOUT>
__global__ void __launch_bounds__(32 * BHMC_MAX_WARPS, 2) k_batch(const SysDev* views, int n_rep, const BatchArgs* args,
                                                                   bhmc_mc_stats* stats) {
  __shared__ MoveStore st;
  __shared__ int rep;
  __shared__ SysDev S;
  init_tables(st.sh, nterms(P));
  bool first = true;
  for (;;) {
    if (threadIdx.x == 0) {
      int r = n_rep;
      if (first && args->n_alone >= 0) r = batch_preferred(args, n_rep);
      if (r < n_rep && atomicExch(&args->claimed[r], 1) != 0) r = n_rep;
      while (r >= n_rep) {  // the largest replica nobody has claimed yet
        const int q = atomicAdd(args->cursor, 1);
        if (q >= n_rep) break;
        const int c = args->order[q];
        if (atomicExch(&args->claimed[c], 1) == 0) r = c;
      }
      rep = r;
    }
    first = false;
    __syncthreads();
    const int r = rep;
    if (r >= n_rep) break;
    if (threadIdx.x == 0) {
      S = views[r];
      st.sh.nxt_m = ~0ULL;
      st.sh.E = *S.energy;
      block_err() = *(volatile int*)S.err != 0;
    }
    __syncthreads();
    const unsigned long long seed = args->seeds[r];
    const uint2 key = make_uint2((unsigned)seed, (unsigned)(seed >> 32));
    bhmc_mc_stats loc;
    loc.moves = loc.accepted = loc.rej_energy = loc.rej_domain = loc.rej_overlap = loc.rej_capacity =
        loc.flagged = 0;
    for (unsigned long long t = 0; t < args->n_moves; ++t) {
      if (block_err()) break;  // every error of the chain is raised by this block
      MoveRec* rec = args->recs ? args->recs + (size_t)r * args->n_moves + t : nullptr;
      const int o = mc_move<P, Real, LAYOUT>(S, st, args->move0 + t, (unsigned)r, key, args->step, rec,
                                             t + 1 < args->n_moves);
      if (o < 0) break;
      if (threadIdx.x == 0) tally(&loc, o, st.sh.result_flagged);
      rdf_sample(S, rdf_points(S, args->move0 + t, args->move0 + t + 1));
    }
    if (threadIdx.x == 0) {
      *S.energy = st.sh.E;
      loc.energy = st.sh.E;
      stats[r] = loc;
      if (args->errs) args->errs[r] = *(volatile int*)S.err;
    }
    __syncthreads();
  }
}


// ---------------------------------------------------------------------------
// Speculative multi-proposal chain: one thread-block cluster of K CTAs runs a
// single chain.  In every step CTA r evaluates trial move m + r against the
// current tree (proposal, rejections, traversal, Metropolis decision,
// capacity rule); after a cluster barrier every CTA reads the K outcomes from
// distributed shared memory.  While no earlier move of the step is accepted
// the tree is the one the sequential chain would see, so the outcomes up to
// and including the first acceptance j are exactly the sequential chain's:
// CTA j commits its move, moves m .. m + j are final, and the chain advances
// by j + 1 (by K when every move was rejected).  The chain, records and
// statistics equal those of K = 1 and of the plain path.

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
// Barrier of every thread of every CTA of the cluster; shared-memory writes
// before it are visible to the cluster's reads after it.
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// *p in the shared memory of CTA `rank` of this cluster.
__device__ __forceinline__ int ld_cluster_int(const int* p, unsigned rank) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  unsigned ra;
  int v;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(ra) : "memory");
  return v;
}

// Trial move m up to its decision, the tree unchanged (all threads of the CTA).
// Returns the outcome, or -1 after a device error (recorded in S.err).
template <int P, typename Real, int LAYOUT>
__device__ int spec_eval(const SysDev& S, MoveStore& st, unsigned long long m, unsigned replica, uint2 key,
                         double step) {
  MoveSh& sh = st.sh;
  if (sh.nxt_m == m) {  // set up during the previous step's commit
    constexpr int n = (int)(sizeof(MoveSetup) / sizeof(int));
    int* dst = reinterpret_cast<int*>(static_cast<MoveSetup*>(&sh));
    const int* src = reinterpret_cast<const int*>(&sh.nxt);
    for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
  } else {
    propose(S, sh, m, replica, key, step, 0);
    __syncthreads();
    setup_roles(S, sh, 0);
    __syncthreads();
    setup_finish(S, sh, 0);
  }
  __syncthreads();
  if (threadIdx.x == 0) sh.nxt_m = ~0ULL;
  if (sh.outcome < 0) {
    eval_move<P, Real, LAYOUT>(S, st, true);
    if (sh.cnt[0][4]) {
      if (threadIdx.x == 0) set_err(S, sh.cnt[0][4]);
      __syncthreads();
      return -1;
    }
    complete_paths(S, sh);
    __syncthreads();
    if (threadIdx.x == 0 && sh.outcome < 0) {
      int acc, fl;
      metropolis(S.beta, sh.dE, sh.alpha, sh.la, acc, fl);
      sh.flagged = fl;
      if (!isfinite(sh.dE)) {
        set_err(S, BHMC_ENONFINITE);
        sh.outcome = BHMC_REJECT_ENERGY;
      } else if (!acc)
        sh.outcome = BHMC_REJECT_ENERGY;
      else if (capacity_violation(S, sh))
        sh.outcome = BHMC_REJECT_CAPACITY;
      else
        sh.outcome = BHMC_ACCEPT;
    }
  }
  __syncthreads();
  return sh.outcome;
}

// One chain of n_moves trial moves from move0 on this cluster of K CTAs (see
// above).  *stats must be zeroed by the caller; recs (may be null) receives
// one record per move.
template <int P, typename Real, int LAYOUT>
__device__ void spec_chain(const SysDev& S, unsigned long long move0, unsigned long long n_moves,
                           unsigned replica, uint2 key, double step, MoveRec* recs, bhmc_mc_stats* stats) {
  __shared__ MoveStore st;
  __shared__ int word;       // this CTA's outcome in the current step (-2: no move, -1: error)
  __shared__ int plan[4];    // first accepted rank, moves made final, error, commit error
  __shared__ int cerr;       // the error word after this CTA's commit
  __shared__ int cion;       // the ion this CTA's commit moved
  MoveSh& sh = st.sh;
  const unsigned rank = cluster_rank(), K = cluster_size();
  // every CTA reads the error word before the barrier, where none of them can
  // have set it yet, so all return together or none does
  const int err0 = *(volatile int*)S.err;
  cluster_sync_all();
  if (err0) return;
  init_tables(sh, S.K);
  if (threadIdx.x == 0) sh.nxt_m = ~0ULL;
  bhmc_mc_stats loc;
  loc.moves = loc.accepted = loc.rej_energy = loc.rej_domain = loc.rej_overlap = loc.rej_capacity =
      loc.flagged = 0;
  unsigned long long done = 0;
  const int warp = threadIdx.x >> 5;
  __syncthreads();
  while (done < n_moves) {
    const bool live = done + rank < n_moves;
    int o = -2;
    if (live) o = spec_eval<P, Real, LAYOUT>(S, st, move0 + done + rank, replica, key, step);
    if (threadIdx.x == 0) word = o;
    cluster_sync_all();
    if (threadIdx.x == 0) {
      int first = (int)K, live_n = 0, bad = 0;
      for (unsigned r = 0; r < K; ++r) {
        const int w = ld_cluster_int(&word, r);
        if (w == -1) bad = 1;
        if (w != -2) ++live_n;
        if (w == BHMC_ACCEPT && first == (int)K) first = (int)r;
      }
      plan[0] = first;
      plan[1] = first < (int)K ? first + 1 : live_n;
      plan[2] = bad;
    }
    __syncthreads();
    const int first = plan[0], nfin = plan[1], bad = plan[2];
    // radial samples of the moves made final before the accepted one (or of
    // all of them) see the tree before the commit: taken by the committing
    // CTA (or CTA 0) before it commits
    const unsigned long long m_step = move0 + done;
    if (!bad && S.rdf_nbins > 0 && (int)rank == (first < (int)K ? first : 0)) {
      rdf_sample(S, rdf_points(S, m_step, m_step + (unsigned long long)(first < (int)K ? first : nfin)));
      __syncthreads();
    }
    // this CTA's trial of the next step, set up while the commit runs (valid
    // unless it draws the ion that the commit moves)
    const unsigned long long mn = move0 + done + (unsigned long long)nfin + rank;
    const bool ahead = !bad && done + (unsigned long long)nfin + rank < n_moves;
    if (!bad && (int)rank < nfin) {
      if (threadIdx.x == 0) {
        tally(&loc, o, sh.flagged);
        if (recs) {
          MoveRec* rec = recs + done + rank;
          rec->i = sh.i;
          rec->r[0] = sh.b[0];
          rec->r[1] = sh.b[1];
          rec->r[2] = sh.b[2];
          rec->dE = sh.dE;
          rec->outcome = sh.outcome;
          rec->flagged = sh.flagged;
        }
      }
    }
    if (!bad && (int)rank == first) {
      const bool split = ahead && blockDim.x == 256;
      if (split && warp >= 5) {  // warps 5-7: the next trial's setup
        propose(S, sh.nxt, mn, replica, key, step, 5);
        bar_ahead();
        setup_roles(S, sh.nxt, 5);
        bar_ahead();
        setup_finish(S, sh.nxt, 5);
        if (threadIdx.x == 160) sh.nxt_m = mn;
      } else {
        commit_move_block(S, st, split ? 160 : 0, split ? 2 : 0);
        if (threadIdx.x == 0) {
          *S.energy += sh.dE;
          cerr = *(volatile int*)S.err;
          cion = (int)sh.i;
        }
      }
    } else if (ahead) {
      propose(S, sh.nxt, mn, replica, key, step, 0);
      __syncthreads();
      setup_roles(S, sh.nxt, 0);
      __syncthreads();
      setup_finish(S, sh.nxt, 0);
      if (threadIdx.x == 0) sh.nxt_m = mn;
    }
    __syncthreads();
    cluster_sync_all();  // the tree is final before the next step, and `word` is read
    if (bad) break;
    if (S.rdf_nbins > 0 && first < (int)K && (int)rank == first)  // the accepted move's own sample
      rdf_sample(S, rdf_points(S, m_step + (unsigned long long)first, m_step + (unsigned long long)first + 1ULL));
    if (threadIdx.x == 0) {
      plan[3] = first < (int)K ? ld_cluster_int(&cerr, (unsigned)first) : 0;
      // a setup that read the moved ion's old position is redone
      if (first < (int)K && sh.nxt_m != ~0ULL && (int)sh.nxt.i == ld_cluster_int(&cion, (unsigned)first))
        sh.nxt_m = ~0ULL;
    }
    __syncthreads();
    if (plan[3]) break;  // the commit failed (pool exhausted): every CTA stops here
    done += (unsigned long long)nfin;
  }
  if (threadIdx.x == 0) {
    atomicAdd(reinterpret_cast<unsigned long long*>(&stats->moves), (unsigned long long)loc.moves);
    atomicAdd(reinterpret_cast<unsigned long long*>(&stats->accepted), (unsigned long long)loc.accepted);
    atomicAdd(reinterpret_cast<unsigned long long*>(&stats->rej_energy), (unsigned long long)loc.rej_energy);
    atomicAdd(reinterpret_cast<unsigned long long*>(&stats->rej_domain), (unsigned long long)loc.rej_domain);
    atomicAdd(reinterpret_cast<unsigned long long*>(&stats->rej_overlap), (unsigned long long)loc.rej_overlap);
    atomicAdd(reinterpret_cast<unsigned long long*>(&stats->rej_capacity), (unsigned long long)loc.rej_capacity);
    atomicAdd(reinterpret_cast<unsigned long long*>(&stats->flagged), (unsigned long long)loc.flagged);
    if (rank == 0) stats->energy = *S.energy;
  }
}

template <int P, typename Real, int LAYOUT>
__global__ void __launch_bounds__(32 * BHMC_MAX_WARPS) k_spec(SysDev S, unsigned long long move0,
                                                             unsigned long long n_moves, unsigned replica,
                                                             uint2 key, double step, MoveRec* recs,
                                                             bhmc_mc_stats* stats) {
  spec_chain<P, Real, LAYOUT>(S, move0, n_moves, replica, key, step, recs, stats);
}

// Replica r of a batch on cluster r (grid = replicas x K CTAs, clusters of K).
template <int P, typename Real, int LAYOUT>
__global__ void __launch_bounds__(32 * BHMC_MAX_WARPS) k_spec_batch(const SysDev* views, int n_rep,
                                                                   const BatchArgs* args, bhmc_mc_stats* stats) {
  __shared__ SysDev S;
  const int r = (int)(blockIdx.x / cluster_size());
  if (r >= n_rep) return;  // the whole cluster
  if (threadIdx.x == 0) S = views[r];
  __syncthreads();
  const unsigned long long seed = args->seeds[r];
  spec_chain<P, Real, LAYOUT>(S, args->move0, args->n_moves, (unsigned)r,
                              make_uint2((unsigned)seed, (unsigned)(seed >> 32)), args->step, nullptr, stats + r);
}

}  // namespace bhmc
