// bhmc_move.cuh -- one Metropolis trial move on the GPU: proposal (Philox),
// rejection tests, energy difference by the fused traversal at the old and new
// positions of the ion and its image (Sec. 1, Sec. 3.2), acceptance (Sec. 2)
// and the local adjustment of the octree (Sec. 3.3) with split/merge.
#pragma once

#include "bhmc_traverse.cuh"

namespace bhmc {

struct MoveSh {
  TravPts T;
  int i, img, npts, nmov;
  double q, qa_img, qb_img;
  double a[3], b[3], ai[3], bi[3];
  int path[4][BHMC_MAX_D + 1];
  int plen[4];
  double part[BHMC_MAX_WARPS];
  int cnt[BHMC_MAX_WARPS][5];
  int outcome, flagged, go;
  double dE, alpha;
  int split_node, split_g;
  float4 tA[BHMC_MAX_C + 2], tB[BHMC_MAX_C + 2];
};

struct MoveStore {
  MoveSh sh;
  WarpStore ws[BHMC_MAX_WARPS];
};

// ---------------------------------------------------------------------------
// Set up a move of ion i to b (thread 0).  Returns -1 to proceed, or the
// rejection outcome (domain / shell), in the oracle's order of tests.
static __device__ int setup_move(const SysDev& S, MoveSh& sh, int i, const double b[3]) {
  sh.i = i;
  sh.q = S.pq[i];
  sh.a[0] = S.px[i];
  sh.a[1] = S.py[i];
  sh.a[2] = S.pz[i];
  for (int k = 0; k < 3; ++k) sh.b[k] = b[k];
  if (!in_root(S, b)) return BHMC_REJECT_DOMAIN;
  if (!shell_ok(S, b)) return BHMC_REJECT_OVERLAP;
  TravPts& T = sh.T;
  sh.npts = 2;
  sh.nmov = 1;
  T.n_excl = 1;
  T.excl[0] = i;
  T.ekey[0] = S.ckey[i];
  T.eq[0] = sh.q;
  for (int k = 0; k < 3; ++k) T.ex[0][k] = sh.a[k];
  if (S.images) {
    const int img = S.n_mob + S.n_fix + i;
    sh.img = img;
    sh.ai[0] = S.px[img];
    sh.ai[1] = S.py[img];
    sh.ai[2] = S.pz[img];
    sh.qa_img = S.pq[img];
    if (!image_of(S, b, sh.q, sh.bi, &sh.qb_img)) return BHMC_REJECT_DOMAIN;
    if (!in_root(S, sh.bi)) return BHMC_REJECT_DOMAIN;
    sh.npts = 4;
    sh.nmov = 2;
    T.n_excl = 2;
    T.excl[1] = img;
    T.ekey[1] = S.ckey[img];
    T.eq[1] = sh.qa_img;
    for (int k = 0; k < 3; ++k) T.ex[1][k] = sh.ai[k];
  }
  const double* pts[4] = {sh.a, sh.b, sh.ai, sh.bi};
  const double w[4] = {-sh.q, sh.q, -sh.qa_img, sh.qb_img};
  for (int s = 0; s < sh.npts; ++s) {
    for (int k = 0; k < 3; ++k) {
      T.x[s][k] = pts[s][k];
      const float2 f = split2(pts[s][k]);
      T.hi[s][k] = f.x;
      T.lo[s][k] = f.y;
    }
    T.w64[s] = w[s];
    T.w[s] = (float)w[s];
  }
  T.pkey[0] = S.ckey[i];
  T.pkey[1] = point_key(S, b[0], b[1], b[2]);
  if (S.images) {
    T.pkey[2] = S.ckey[sh.img];
    T.pkey[3] = point_key(S, sh.bi[0], sh.bi[1], sh.bi[2]);
  }
  return -1;
}

__device__ __forceinline__ unsigned warp_points(int warp, int W, int npts) {
  if (W == 1) return npts == 4 ? 15u : 3u;
  if (W == 2) return npts == 4 ? (warp == 0 ? 3u : 12u) : (1u << warp);
  return warp < npts ? (1u << warp) : 0u;
}

// All warps: traverse, then thread 0 assembles dE (FP64).  Requires a
// __syncthreads() after setup.  Returns with sh.dE and sh.cnt filled.
template <int P, typename Real, int LAYOUT>
__device__ void eval_move(const SysDev& S, MoveStore& st, bool record_path) {
  MoveSh& sh = st.sh;
  const int warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  for (int k = threadIdx.x; k < 4 * (BHMC_MAX_D + 1); k += blockDim.x) (&sh.path[0][0])[k] = -1;
  __syncthreads();
  const unsigned pm = warp_points(warp, W, sh.npts);
  TravOut o;
  o.sum = 0.0;
  o.visited = o.accepted = o.pairs = o.fp64 = o.err = 0;
  if (pm) warp_traverse<P, Real, LAYOUT>(S, sh.T, st.ws[warp], pm, record_path ? sh.path : nullptr, o);
  if ((threadIdx.x & 31) == 0) {
    sh.part[warp] = o.sum;
    sh.cnt[warp][0] = o.visited;
    sh.cnt[warp][1] = o.accepted;
    sh.cnt[warp][2] = o.pairs;
    sh.cnt[warp][3] = o.fp64;
    sh.cnt[warp][4] = o.err;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < W; ++w) s += sh.part[w];
    if (sh.npts == 4) {
      double pb, pa;
      if (sizeof(Real) == 4) {
        const float2 bx = split2(sh.b[0]), by = split2(sh.b[1]), bz = split2(sh.b[2]);
        const float2 ix = split2(sh.bi[0]), iy = split2(sh.bi[1]), iz = split2(sh.bi[2]);
        const float2 ax = split2(sh.a[0]), ay = split2(sh.a[1]), az = split2(sh.a[2]);
        const float2 jx = split2(sh.ai[0]), jy = split2(sh.ai[1]), jz = split2(sh.ai[2]);
        float dx = (bx.x - ix.x) + (bx.y - ix.y), dy = (by.x - iy.x) + (by.y - iy.y),
              dz = (bz.x - iz.x) + (bz.y - iz.y);
        pb = (double)((float)(sh.q * sh.qb_img) * rsqrtf(dx * dx + dy * dy + dz * dz));
        dx = (ax.x - jx.x) + (ax.y - jx.y);
        dy = (ay.x - jy.x) + (ay.y - jy.y);
        dz = (az.x - jz.x) + (az.y - jz.y);
        pa = (double)((float)(sh.q * sh.qa_img) * rsqrtf(dx * dx + dy * dy + dz * dz));
      } else {
        double dx = sh.b[0] - sh.bi[0], dy = sh.b[1] - sh.bi[1], dz = sh.b[2] - sh.bi[2];
        pb = sh.q * sh.qb_img / sqrt(dx * dx + dy * dy + dz * dz);
        dx = sh.a[0] - sh.ai[0];
        dy = sh.a[1] - sh.ai[1];
        dz = sh.a[2] - sh.ai[2];
        pa = sh.q * sh.qa_img / sqrt(dx * dx + dy * dy + dz * dz);
      }
      s += pb - pa;
    }
    sh.dE = S.lB * s;
    for (int w = 1; w < W; ++w)
      for (int k = 0; k < 5; ++k)
        sh.cnt[0][k] = (k == 4) ? max(sh.cnt[0][k], sh.cnt[w][k]) : sh.cnt[0][k] + sh.cnt[w][k];
  }
  __syncthreads();
}

// Complete the cluster paths of the four points by descending from the deepest
// recorded cluster (threads 0..npts-1).
static __device__ void complete_paths(const SysDev& S, MoveSh& sh) {
  const int s = threadIdx.x;
  if (s < sh.npts) {
    int d = 0;
    if (sh.path[s][0] < 0) sh.path[s][0] = 0;
    while (d < S.Dmax && sh.path[s][d + 1] >= 0) ++d;
    int node = sh.path[s][d];
    for (;;) {
      const int fc = S.nB[node].x;
      if (fc < 0 || d >= S.Dmax) break;
      const int o = (int)((sh.T.pkey[s] >> (3 * (S.Dmax - d - 1))) & 7ULL);
      node = fc + o;
      ++d;
      sh.path[s][d] = node;
    }
    sh.plen[s] = d;
  }
}

// Capacity rule (thread 0): after the move no depth-Dmax cell may hold more than C charges.
static __device__ bool capacity_violation(const SysDev& S, const MoveSh& sh) {
  for (int s = 1; s < sh.npts; s += 2) {
    const unsigned long long kb = sh.T.pkey[s];
    const int L = sh.path[s][sh.plen[s]];
    const int c = S.nB[L].y;
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

// Local adjustment (Sec. 3.3) of an accepted move, all threads of the block.
// Requires complete paths (complete_paths) and sh.T.pkey of the new points.
static __device__ void commit_move_block(const SysDev& S, MoveSh& sh) {
  const int K = S.K, SC = S.C + 2;
  // (A) FP64 moments on both paths, per level: same cluster -> M += mb - ma,
  // else M_old -= ma and M_new += mb.
  for (int m = 0; m < sh.nmov; ++m) {
    const int pa = 2 * m, pb = 2 * m + 1;
    const int La = sh.plen[pa], Lb = sh.plen[pb];
    const int Dn = max(La, Lb) + 1;
    const double qa = m ? sh.qa_img : sh.q, qb = m ? sh.qb_img : sh.q;
    const double* A_ = m ? sh.ai : sh.a;
    const double* B_ = m ? sh.bi : sh.b;
    for (int it = threadIdx.x; it < Dn * K; it += blockDim.x) {
      const int d = it / K, t = it - d * K;
      const int na = d <= La ? sh.path[pa][d] : -1;
      const int nb = d <= Lb ? sh.path[pb][d] : -1;
      int n1, n2, n3;
      term_exponents(t, n1, n2, n3);
      if (na >= 0 && na == nb) {
        const float4 c = S.nA[na];
        const double ma = mono_term(n1, n2, n3, qa, __dsub_rn(A_[0], (double)c.x),
                                    __dsub_rn(A_[1], (double)c.y), __dsub_rn(A_[2], (double)c.z));
        const double mb = mono_term(n1, n2, n3, qb, __dsub_rn(B_[0], (double)c.x),
                                    __dsub_rn(B_[1], (double)c.y), __dsub_rn(B_[2], (double)c.z));
        double* M = &S.M64[(size_t)na * K + t];
        *M = __dadd_rn(*M, __dsub_rn(mb, ma));
        mirror(S, na, t, *M);
      } else {
        if (na >= 0) {
          const float4 c = S.nA[na];
          const double ma = mono_term(n1, n2, n3, qa, __dsub_rn(A_[0], (double)c.x),
                                      __dsub_rn(A_[1], (double)c.y), __dsub_rn(A_[2], (double)c.z));
          double* M = &S.M64[(size_t)na * K + t];
          *M = __dsub_rn(*M, ma);
          mirror(S, na, t, *M);
        }
        if (nb >= 0) {
          const float4 c = S.nA[nb];
          const double mb = mono_term(n1, n2, n3, qb, __dsub_rn(B_[0], (double)c.x),
                                      __dsub_rn(B_[1], (double)c.y), __dsub_rn(B_[2], (double)c.z));
          double* M = &S.M64[(size_t)nb * K + t];
          *M = __dadd_rn(*M, mb);
          mirror(S, nb, t, *M);
        }
      }
    }
    __syncthreads();
  }
  // (B) counts, leaf slots (delete = refill with the last slot, add = append), tracking
  if (threadIdx.x == 0) {
    for (int m = 0; m < sh.nmov; ++m) {
      const int pa = 2 * m, pb = 2 * m + 1;
      const int La = sh.plen[pa], Lb = sh.plen[pb];
      const int j = m ? sh.img : sh.i;
      const double* B_ = m ? sh.bi : sh.b;
      const double qb = m ? sh.qb_img : sh.q;
      for (int d = 0; d <= max(La, Lb); ++d) {
        const int na = d <= La ? sh.path[pa][d] : -1;
        const int nb = d <= Lb ? sh.path[pb][d] : -1;
        if (na != nb) {
          if (na >= 0) *count_ptr(S, na) -= 1;
          if (nb >= 0) *count_ptr(S, nb) += 1;
        }
      }
      const float2 fx = split2(B_[0]), fy = split2(B_[1]), fz = split2(B_[2]);
      const float4 na4 = make_float4(fx.x, fy.x, fz.x, (float)qb);
      const float4 nb4 = make_float4(fx.y, fy.y, fz.y, __int_as_float(j));
      const int LA = sh.path[pa][La], LB = sh.path[pb][Lb];
      if (LA == LB) {
        const int k = S.slot_of[j];
        S.sA[LA * SC + k] = na4;
        S.sB[LA * SC + k] = nb4;
      } else {
        const int k = S.slot_of[j];
        const int last = S.nB[LA].y;
        if (k != last) {
          const float4 la = S.sA[LA * SC + last], lb = S.sB[LA * SC + last];
          S.sA[LA * SC + k] = la;
          S.sB[LA * SC + k] = lb;
          S.slot_of[__float_as_int(lb.w)] = k;
        }
        const int kk = S.nB[LB].y - 1;
        S.sA[LB * SC + kk] = na4;
        S.sB[LB * SC + kk] = nb4;
        S.leaf_of[j] = LB;
        S.slot_of[j] = kk;
      }
      S.px[j] = B_[0];
      S.py[j] = B_[1];
      S.pz[j] = B_[2];
      S.pq[j] = qb;
      S.ckey[j] = sh.T.pkey[pb];
    }
    // (C) merge the topmost internal cluster on an old path holding <= C charges
    for (int m = 0; m < sh.nmov; ++m) {
      const int pa = 2 * m;
      for (int d = 0; d <= sh.plen[pa]; ++d) {
        const int A = sh.path[pa][d];
        if (d > 0 && S.nB[sh.path[pa][d - 1]].x != (A & ~7)) break;
        const int4 b = S.nB[A];
        if (b.x < 0) break;
        if (b.y <= S.C) {
          merge_cluster(S, sh, A);
          break;
        }
      }
    }
  }
  __syncthreads();
  // (D) split the new leaves while they hold more than C charges
  for (int m = 0; m < sh.nmov; ++m) {
    const int j = m ? sh.img : sh.i;
    for (int guard = 0; guard <= BHMC_MAX_D; ++guard) {
      if (threadIdx.x == 0) {
        const int L = S.leaf_of[j];
        const int4 b = S.nB[L];
        const unsigned long long key = ((unsigned long long)(unsigned)b.w << 32) | (unsigned)b.z;
        const int dL = key_depth(key);
        sh.split_node = -1;
        if (b.y > S.C && dL < S.Dmax) {
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
      __syncthreads();
      if (sh.split_node < 0) break;
      for (int it = threadIdx.x; it < 8 * K; it += blockDim.x) {
        const int o = it / K, t = it - o * K;
        const int ch = sh.split_g + o;
        const float4 c = S.nA[ch];
        const int cnt = S.nB[ch].y;
        int n1, n2, n3;
        term_exponents(t, n1, n2, n3);
        double M = 0.0;
        for (int k = 0; k < cnt; ++k) {
          const int idx = __float_as_int(S.sB[ch * SC + k].w);
          M = __dadd_rn(M, mono_term(n1, n2, n3, S.pq[idx], __dsub_rn(S.px[idx], (double)c.x),
                                     __dsub_rn(S.py[idx], (double)c.y), __dsub_rn(S.pz[idx], (double)c.z)));
        }
        S.M64[(size_t)ch * K + t] = M;
        mirror(S, ch, t, M);
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// Metropolis decision in FP64 (alpha <= exp(-beta dE)), settled in FP32 when
// the two sides differ by more than a safe margin.
__device__ __forceinline__ void metropolis(double beta, double dE, double alpha, int& accept,
                                           int& flagged) {
  const double x = -beta * dE;
  const float xf = (float)x, la = logf((float)alpha);
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

// One full trial move m of a chain (all threads).  Returns the outcome.
template <int P, typename Real, int LAYOUT>
__device__ int mc_move(const SysDev& S, MoveStore& st, unsigned long long m, unsigned replica,
                       uint2 key, double step, MoveRec* rec) {
  MoveSh& sh = st.sh;
  if (threadIdx.x == 0) {
    const uint4 u = philox(make_uint4((unsigned)m, (unsigned)(m >> 32), replica, 0u), key);
    const uint4 v = philox(make_uint4((unsigned)m, (unsigned)(m >> 32), replica, 1u), key);
    const int i = (int)(((unsigned long long)u.x * (unsigned long long)S.n_mob) >> 32);
    const unsigned uu[3] = {u.y, u.z, u.w};
    double b[3];
    const double src[3] = {S.px[i], S.py[i], S.pz[i]};
    for (int k = 0; k < 3; ++k) {
      const double delta =
          __dmul_rn(__dsub_rn(__dadd_rn(__dmul_rn((double)uu[k], 0x1p-32), 0x1p-33), 0.5), step);
      b[k] = __dadd_rn(src[k], delta);
    }
    sh.outcome = setup_move(S, sh, i, b);
    sh.dE = 0.0;
    sh.flagged = 0;
    sh.alpha = __dmul_rn(__dadd_rn((double)v.x, 0.5), 0x1p-32);
    sh.go = (sh.outcome < 0);
  }
  __syncthreads();
  if (sh.go) {
    eval_move<P, Real, LAYOUT>(S, st, true);
    if (sh.cnt[0][4]) {
      if (threadIdx.x == 0) set_err(S, sh.cnt[0][4]);
      return -1;
    }
    complete_paths(S, sh);
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc, fl;
      metropolis(S.beta, sh.dE, sh.alpha, acc, fl);
      sh.flagged = fl;
      if (!acc)
        sh.outcome = BHMC_REJECT_ENERGY;
      else if (capacity_violation(S, sh))
        sh.outcome = BHMC_REJECT_CAPACITY;
      else
        sh.outcome = BHMC_ACCEPT;
    }
    __syncthreads();
    if (sh.outcome == BHMC_ACCEPT) {
      commit_move_block(S, sh);
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
__global__ void __launch_bounds__(128) k_delta(SysDev S, int i, double bx, double by, double bz,
                                               DeltaOut* out) {
  __shared__ MoveStore st;
  if (threadIdx.x == 0) {
    const double b[3] = {bx, by, bz};
    const int o = setup_move(S, st.sh, i, b);
    st.sh.go = o < 0;
    out->status = o < 0 ? 0 : (o == BHMC_REJECT_DOMAIN ? BHMC_EDOMAIN : BHMC_EOVERLAP);
  }
  __syncthreads();
  if (!st.sh.go) return;
  eval_move<P, Real, LAYOUT>(S, st, false);
  if (threadIdx.x == 0) {
    out->dE = st.sh.dE;
    for (int k = 0; k < 4; ++k) out->cnt[k] = st.sh.cnt[0][k];
    out->err = st.sh.cnt[0][4];
  }
}

template <int P, typename Real, int LAYOUT>
__global__ void __launch_bounds__(128) k_step(SysDev S, unsigned long long m, unsigned replica,
                                              uint2 key, double step, MoveRec* recs,
                                              bhmc_mc_stats* stats) {
  __shared__ MoveStore st;
  if (*(volatile int*)S.err) return;
  const int o = mc_move<P, Real, LAYOUT>(S, st, m, replica, key, step, recs);
  if (threadIdx.x == 0 && o >= 0) {
    tally(stats, o, st.sh.flagged);
    stats->energy = *S.energy;
  }
}

struct BatchArgs {
  unsigned long long n_moves, move0;
  double step;
  const unsigned long long* seeds;
};

template <int P, typename Real, int LAYOUT>
__global__ void __launch_bounds__(128) k_batch(const SysDev* views, int n_rep, const BatchArgs* args,
                                               int* next, bhmc_mc_stats* stats) {
  __shared__ MoveStore st;
  __shared__ int rep;
  __shared__ SysDev S;
  for (;;) {
    if (threadIdx.x == 0) rep = atomicAdd(next, 1);
    __syncthreads();
    const int r = rep;
    if (r >= n_rep) break;
    if (threadIdx.x == 0) S = views[r];
    __syncthreads();
    const unsigned long long seed = args->seeds[r];
    const uint2 key = make_uint2((unsigned)seed, (unsigned)(seed >> 32));
    bhmc_mc_stats loc;
    loc.moves = loc.accepted = loc.rej_energy = loc.rej_domain = loc.rej_overlap = loc.rej_capacity =
        loc.flagged = 0;
    for (unsigned long long t = 0; t < args->n_moves; ++t) {
      if (*(volatile int*)S.err) break;
      const int o = mc_move<P, Real, LAYOUT>(S, st, args->move0 + t, (unsigned)r, key, args->step,
                                             nullptr);
      if (o < 0) break;
      if (threadIdx.x == 0) tally(&loc, o, st.sh.flagged);
    }
    if (threadIdx.x == 0) {
      loc.energy = *S.energy;
      stats[r] = loc;
    }
    __syncthreads();
  }
}

// Full treecode energy: one warp per target charge j, S = {j}.
template <int P, typename Real, int LAYOUT>
__global__ void __launch_bounds__(128) k_energy(SysDev S, double* partial, int* err) {
  __shared__ TravPts Tw[BHMC_MAX_WARPS];
  __shared__ WarpStore ws[BHMC_MAX_WARPS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int W = blockDim.x >> 5;
  double acc = 0.0;
  for (int j = blockIdx.x * W + warp; j < S.n_tot; j += gridDim.x * W) {
    TravPts& T = Tw[warp];
    if (lane == 0) {
      const double x[3] = {S.px[j], S.py[j], S.pz[j]};
      for (int k = 0; k < 3; ++k) {
        T.x[0][k] = x[k];
        const float2 f = split2(x[k]);
        T.hi[0][k] = f.x;
        T.lo[0][k] = f.y;
      }
      T.w[0] = 1.0f;
      T.w64[0] = 1.0;
      T.pkey[0] = 0ULL;
      T.n_excl = 1;
      T.excl[0] = j;
      T.ekey[0] = S.ckey[j];
      T.eq[0] = S.pq[j];
      T.ex[0][0] = x[0];
      T.ex[0][1] = x[1];
      T.ex[0][2] = x[2];
    }
    __syncwarp();
    TravOut o;
    warp_traverse<P, Real, LAYOUT>(S, T, ws[warp], 1u, nullptr, o);
    if (o.err && lane == 0) atomicCAS(err, 0, o.err);
    acc += S.pq[j] * o.sum;
    __syncwarp();
  }
  if (lane == 0) partial[blockIdx.x * W + warp] = acc;
}

}  // namespace bhmc
