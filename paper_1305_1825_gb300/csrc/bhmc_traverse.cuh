// bhmc_traverse.cuh -- warp-cooperative octree traversal (Sec. 3.2) evaluating
// the potential of the tree minus an excluded set at up to four points at once.
//
// Each lane examines one cluster; a round pops up to four groups of eight
// siblings from a per-warp stack in shared memory.  A stack entry carries two
// 4-bit masks over the evaluation points: `open` (regular traversal: MAC test,
// then multipole / open / direct) and `forced` (inside a cluster that failed the
// MAC with N'_A <= N_0: direct over all its particles, no MAC).  The MAC
// decision of every (cluster, point) pair is the FP64 decision
// rho_A^2 <= theta^2 ((dx*dx + dy*dy) + dz*dz): FP32 settles it when the value
// is further than 2^-17 (relative) from the threshold, the exact FP64 sequence
// otherwise.
#pragma once

#include "bhmc_common.cuh"
#include "bhmc_taylor.cuh"

namespace bhmc {

struct TravPts {
  double x[4][3];          // evaluation points (FP64)
  float hi[4][3], lo[4][3];// x = hi + lo
  float w[4];              // weight of each point's potential in the sum
  double w64[4];
  unsigned long long pkey[4];  // depth-Dmax key of each point (path recording)
  int n_excl;
  int excl[2];             // excluded charges (still in the tree)
  unsigned long long ekey[2];
  double eq[2];
  double ex[2][3];
  float ehi[2][3], elo[2][3];  // excluded positions as float pairs
  float eqf[2];
  float4 h4[4], l4[4];         // the points' float pairs as vectors (w unused)
};

struct WarpStore {
  uint2 stk[BHMC_STACK];
  unsigned mi[128];        // multipole items: node << 4 | excluded-inside mask << 2 | point
  uint2 di[32];            // direct items: {leaf, count << 4 | point mask}
};

struct TravOut {
  double sum;
  int visited, accepted, pairs, fp64;
  int err;
};

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <typename Real>
__device__ __forceinline__ bool mac_test(const SysDev& S, const float4& a, const TravPts& T, int s,
                                         int& fp64);

template <>
__device__ __forceinline__ bool mac_test<float>(const SysDev& S, const float4& a, const TravPts& T,
                                                int s, int& fp64) {
  const float rx = (a.x - T.hi[s][0]) - T.lo[s][0];
  const float ry = (a.y - T.hi[s][1]) - T.lo[s][1];
  const float rz = (a.z - T.hi[s][2]) - T.lo[s][2];
  const float d2 = rx * rx + ry * ry + rz * rz;
  const float rho2 = 3.0f * a.w * a.w;
  const float t = S.theta2f * d2;
  if (t >= rho2 * 1.0000076293945312f) return true;   // 1 + 2^-17
  if (t <= rho2 * 0.9999923706054688f) return false;  // 1 - 2^-17
  ++fp64;
  const double dx = __dsub_rn((double)a.x, T.x[s][0]);
  const double dy = __dsub_rn((double)a.y, T.x[s][1]);
  const double dz = __dsub_rn((double)a.z, T.x[s][2]);
  const double dd = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  const double r2 = __dmul_rn(__dmul_rn(3.0, (double)a.w), (double)a.w);
  return r2 <= __dmul_rn(S.theta2, dd);
}

template <>
__device__ __forceinline__ bool mac_test<double>(const SysDev& S, const float4& a,
                                                 const TravPts& T, int s, int& fp64) {
  const double dx = __dsub_rn((double)a.x, T.x[s][0]);
  const double dy = __dsub_rn((double)a.y, T.x[s][1]);
  const double dz = __dsub_rn((double)a.z, T.x[s][2]);
  const double dd = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  const double r2 = __dmul_rn(__dmul_rn(3.0, (double)a.w), (double)a.w);
  return r2 <= __dmul_rn(S.theta2, dd);
}

// sum_n T_n d^n for a point at offset d from the cluster centre: the p-th
// order expansion of 1/|x - r| for a single charge.
template <int P, typename R>
__device__ __forceinline__ R dot_monomials(const R (&T)[nterms(P)], R dx, R dy, R dz) {
  R px[P + 1], py[P + 1], pz[P + 1];
  px[0] = py[0] = pz[0] = R(1);
#pragma unroll
  for (int k = 1; k <= P; ++k) {
    px[k] = px[k - 1] * dx;
    py[k] = py[k - 1] * dy;
    pz[k] = pz[k - 1] * dz;
  }
  R v = R(0);
#pragma unroll
  for (int k = 0; k <= P; ++k)
#pragma unroll
    for (int n1 = k; n1 >= 0; --n1)
#pragma unroll
      for (int n2 = k - n1; n2 >= 0; --n2) v += T[tidx(n1, n2, k - n1 - n2)] * (px[n1] * py[n2] * pz[k - n1 - n2]);
  return v;
}

// Multipole term of cluster `node` at point s: sum_n T_n(r_A - x) M'_n with
// M' = M minus the terms of the excluded charges inside the cluster (emask);
// the excluded charges' own expansions are subtracted explicitly.
template <int P, typename Real, int LAYOUT>
__device__ __forceinline__ Real eval_item(const SysDev& S, const TravPts& T, int node, int s,
                                          unsigned emask) {
  constexpr int K = nterms(P);
  const float4 a = S.nA[node];
  if (sizeof(Real) == 4) {
    const float rx = (a.x - T.hi[s][0]) - T.lo[s][0];
    const float ry = (a.y - T.hi[s][1]) - T.lo[s][1];
    const float rz = (a.z - T.hi[s][2]) - T.lo[s][2];
    float Tc[K];
    taylor<P, float>(rx, ry, rz, Tc);
    float v = 0.f;
    if (LAYOUT == BHMC_LAYOUT_AOS) {
      constexpr int KP = pad4(K);
      const float4* M4 = reinterpret_cast<const float4*>(S.M32 + (size_t)node * KP);
#pragma unroll
      for (int t4 = 0; t4 < KP / 4; ++t4) {
        const float4 m = M4[t4];
        const float mm[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (4 * t4 + u < K) v = fmaf(Tc[4 * t4 + u], mm[u], v);
      }
    } else {
      const float* M = S.M32 + node;
#pragma unroll
      for (int t = 0; t < K; ++t) v = fmaf(Tc[t], M[(size_t)t * S.node_cap], v);
    }
    while (emask) {
      const int k = __ffs(emask) - 1;
      emask &= emask - 1;
      const float dx = (T.ehi[k][0] - a.x) + T.elo[k][0];
      const float dy = (T.ehi[k][1] - a.y) + T.elo[k][1];
      const float dz = (T.ehi[k][2] - a.z) + T.elo[k][2];
      v -= T.eqf[k] * dot_monomials<P, float>(Tc, dx, dy, dz);
    }
    return (Real)v;
  } else {
    const double rx = __dsub_rn((double)a.x, T.x[s][0]);
    const double ry = __dsub_rn((double)a.y, T.x[s][1]);
    const double rz = __dsub_rn((double)a.z, T.x[s][2]);
    double Tc[K];
    taylor<P, double>(rx, ry, rz, Tc);
    const double* M = S.M64 + (size_t)node * K;
    double v = 0.0;
#pragma unroll
    for (int t = 0; t < K; ++t) v += Tc[t] * M[t];
    while (emask) {
      const int k = __ffs(emask) - 1;
      emask &= emask - 1;
      v -= T.eq[k] * dot_monomials<P, double>(Tc, __dsub_rn(T.ex[k][0], (double)a.x),
                                               __dsub_rn(T.ex[k][1], (double)a.y),
                                               __dsub_rn(T.ex[k][2], (double)a.z));
    }
    return (Real)v;
  }
}

// Kahan-compensated accumulation in FP32; plain in FP64.
template <typename Real>
struct Acc;
template <>
struct Acc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double value() const { return s; }
};

// Direct terms of one leaf slot against the points of `m`.
template <typename Real>
__device__ __forceinline__ void direct_slot(const SysDev& S, const TravPts& T, float4 sa, float4 sb,
                                            unsigned m, Acc<Real>& acc, int& pairs) {
  const int j = __float_as_int(sb.w);
  for (int u = 0; u < T.n_excl; ++u)
    if (T.excl[u] == j) return;
  while (m) {
    const int s = __ffs(m) - 1;
    m &= m - 1;
    if (sizeof(Real) == 4) {
      const float dx = (sa.x - T.hi[s][0]) + (sb.x - T.lo[s][0]);
      const float dy = (sa.y - T.hi[s][1]) + (sb.y - T.lo[s][1]);
      const float dz = (sa.z - T.hi[s][2]) + (sb.z - T.lo[s][2]);
      const float r2 = dx * dx + dy * dy + dz * dz;
      acc.add((Real)(T.w[s] * (sa.w * rsqrtf(r2))));
    } else {
      const double dx = __dsub_rn(S.px[j], T.x[s][0]);
      const double dy = __dsub_rn(S.py[j], T.x[s][1]);
      const double dz = __dsub_rn(S.pz[j], T.x[s][2]);
      const double r = sqrt(dx * dx + dy * dy + dz * dz);
      acc.add((Real)(T.w64[s] * (S.pq[j] / r)));
    }
    ++pairs;
  }
}

// Traverse from the root for the points in `pmask`; `path` (may be null)
// receives, per point and level, the cluster containing the point.  The
// headers of the next round's clusters are loaded before the current round's
// multipole and direct terms are evaluated, so their latency overlaps compute.
template <int P, typename Real, int LAYOUT>
__device__ void warp_traverse(const SysDev& S, const TravPts& T, WarpStore& W, unsigned pmask,
                              int (*path)[BHMC_MAX_D + 1], TravOut& out) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int g = lane >> 3;
  Acc<Real> acc;
  int visited = 0, accepted = 0, pairs = 0, fp64 = 0, err = 0;
  int cp = 1;
  while (cp < S.C) cp <<= 1;
  const int lg = 31 - __clz(cp);
  const int SC = S.C + 2;
  // first round: the root group {root, 7 empty slots}
  int top = 0;
  int npop = 1;
  uint2 e = make_uint2(0u, g == 0 ? pmask : 0u);
  int4 b = make_int4(-1, 0, 0, 0);
  float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
  if (g == 0) {
    b = S.nB[lane & 7];
    a = S.nA[lane & 7];
  }
  int rounds = 0;
  while (npop > 0) {
    if (++rounds > (1 << 22)) {
      err = BHMC_ETIMEOUT;
      break;
    }
    const int node = (int)e.x + (lane & 7);
    const unsigned om = e.y & 15u, fd = (e.y >> 4) & 15u;
    unsigned mac = 0, open = 0, fdc = 0, dir = 0, emask = 0;
    int fc = -1, cnt = 0;
    const unsigned long long key = ((unsigned long long)(unsigned)b.w << 32) | (unsigned)b.z;
    if (g < npop && (om | fd) && key != 0ULL) {
      fc = b.x;
      cnt = b.y;
      const int d = key_depth(key);
      const int sh = 3 * (S.Dmax - d);
      for (int k = 0; k < T.n_excl; ++k) emask |= ((T.ekey[k] >> sh) == key) ? (1u << k) : 0u;
      if (path) {
        unsigned all = om | fd;
        while (all) {
          const int s = __ffs(all) - 1;
          all &= all - 1;
          if ((T.pkey[s] >> sh) == key) path[s][d] = node;
        }
      }
      visited += __popc(om);
      const int np = cnt - __popc(emask);
      if (np > 0) {
        unsigned m = om;
        while (m) {
          const int s = __ffs(m) - 1;
          m &= m - 1;
          const unsigned bit = 1u << s;
          if (np >= S.N0 && mac_test<Real>(S, a, T, s, fp64))
            mac |= bit;
          else if (fc >= 0)
            (np > S.N0 ? open : fdc) |= bit;
          else
            dir |= bit;
        }
        if (fd) {
          if (fc >= 0)
            fdc |= fd;
          else
            dir |= fd;
        }
      }
    }
    // children to the stack (the popped entries' slots are reused)
    const bool push = (open | fdc) != 0;
    const unsigned pb = __ballot_sync(FULL, push);
    const int npush = __popc(pb);
    if (top + npush > BHMC_STACK) {
      err = BHMC_ESTACK;
      break;
    }
    if (push) W.stk[top + __popc(pb & lanemask_lt())] = make_uint2((unsigned)fc, open | (fdc << 4));
    top += npush;
    // multipole and direct items of this round
    const int nm = __popc(mac);
    int incl = nm;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    {
      int pos = incl - nm;
      unsigned m = mac;
      while (m) {
        const int s = __ffs(m) - 1;
        m &= m - 1;
        W.mi[pos++] = ((unsigned)node << 4) | (emask << 2) | (unsigned)s;
      }
    }
    accepted += nm;
    const unsigned db = __ballot_sync(FULL, dir != 0);
    const int ndir = __popc(db);
    if (dir) W.di[__popc(db & lanemask_lt())] = make_uint2((unsigned)node, ((unsigned)cnt << 4) | dir);
    __syncwarp();
    // next round: pop and prefetch its headers
    const int npop_n = min(top, 4);
    uint2 e_n = make_uint2(0u, 0u);
    int4 b_n = make_int4(-1, 0, 0, 0);
    float4 a_n = make_float4(0.f, 0.f, 0.f, 0.f);
    if (g < npop_n) {
      e_n = W.stk[top - 1 - g];
      const int nn = (int)e_n.x + (lane & 7);
      b_n = S.nB[nn];
      a_n = S.nA[nn];
    }
    top -= npop_n;
    // first direct pass: issue its loads before the multipole work
    const int per = 32 >> lg;
    const int kk = lane & (cp - 1);
    uint2 di0 = make_uint2(0u, 0u);
    float4 sa0 = make_float4(0.f, 0.f, 0.f, 0.f), sb0 = sa0;
    bool have0 = false;
    if ((lane >> lg) < ndir) {
      di0 = W.di[lane >> lg];
      if (kk < (int)(di0.y >> 4)) {
        const int slot = (int)di0.x * SC + kk;
        sa0 = S.sA[slot];
        sb0 = S.sB[slot];
        have0 = true;
      }
    }
    for (int k = lane; k < total; k += 32) {
      const unsigned it = W.mi[k];
      const int s = (int)(it & 3u);
      const Real v = eval_item<P, Real, LAYOUT>(S, T, (int)(it >> 4), s, (it >> 2) & 3u);
      acc.add(sizeof(Real) == 4 ? (Real)(T.w[s] * (float)v) : (Real)(T.w64[s] * (double)v));
    }
    if (have0) direct_slot<Real>(S, T, sa0, sb0, di0.y & 15u, acc, pairs);
    for (int base = per; base < ndir; base += per) {
      const int item = base + (lane >> lg);
      if (item < ndir) {
        const uint2 di = W.di[item];
        if (kk < (int)(di.y >> 4)) {
          const int slot = (int)di.x * SC + kk;
          direct_slot<Real>(S, T, S.sA[slot], S.sB[slot], di.y & 15u, acc, pairs);
        }
      }
    }
    __syncwarp();
    e = e_n;
    b = b_n;
    a = a_n;
    npop = npop_n;
  }
  double v = acc.value();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  out.sum = v;
  out.visited = __reduce_add_sync(FULL, visited);
  out.accepted = __reduce_add_sync(FULL, accepted);
  out.pairs = __reduce_add_sync(FULL, pairs);
  out.fp64 = __reduce_add_sync(FULL, fp64);
  out.err = __reduce_max_sync(FULL, err);
}

}  // namespace bhmc
