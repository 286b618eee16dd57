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
};

struct WarpStore {
  uint2 stk[BHMC_STACK];
  unsigned mi[128];        // multipole items: node << 3 | corrected << 2 | point
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

// Moments of `node` minus the terms of the excluded charges inside it (FP64).
static __device__ __noinline__ void corrected_moments(const SysDev& S, const TravPts& T, int node,
                                               double* M) {
  const float4 a = S.nA[node];
  const int4 b = S.nB[node];
  const unsigned long long key = ((unsigned long long)(unsigned)b.w << 32) | (unsigned)b.z;
  const int sh = 3 * (S.Dmax - key_depth(key));
  for (int t = 0; t < S.K; ++t) M[t] = S.M64[(size_t)node * S.K + t];
  for (int k = 0; k < T.n_excl; ++k) {
    if ((T.ekey[k] >> sh) != key) continue;
    const double dx = __dsub_rn(T.ex[k][0], (double)a.x);
    const double dy = __dsub_rn(T.ex[k][1], (double)a.y);
    const double dz = __dsub_rn(T.ex[k][2], (double)a.z);
    for (int t = 0; t < S.K; ++t) {
      int n1, n2, n3;
      term_exponents(t, n1, n2, n3);
      M[t] = __dsub_rn(M[t], mono_term(n1, n2, n3, T.eq[k], dx, dy, dz));
    }
  }
}

template <int P, typename Real, int LAYOUT>
__device__ __forceinline__ Real eval_item(const SysDev& S, const TravPts& T, int node, int s,
                                          bool corr) {
  const float4 a = S.nA[node];
  if (sizeof(Real) == 4) {
    const float rx = (a.x - T.hi[s][0]) - T.lo[s][0];
    const float ry = (a.y - T.hi[s][1]) - T.lo[s][1];
    const float rz = (a.z - T.hi[s][2]) - T.lo[s][2];
    if (!corr) return (Real)multipole_f32<P, LAYOUT>(S, node, rx, ry, rz);
    double M[nterms(P)];
    corrected_moments(S, T, node, M);
    return (Real)multipole_explicit<P, float>(rx, ry, rz, M);
  } else {
    const double rx = __dsub_rn((double)a.x, T.x[s][0]);
    const double ry = __dsub_rn((double)a.y, T.x[s][1]);
    const double rz = __dsub_rn((double)a.z, T.x[s][2]);
    if (!corr) return (Real)multipole_f64<P>(S, node, rx, ry, rz);
    double M[nterms(P)];
    corrected_moments(S, T, node, M);
    return (Real)multipole_explicit<P, double>(rx, ry, rz, M);
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

// Traverse from the root for the points in `pmask`; `path` (may be null)
// receives, per point and level, the cluster containing the point.
template <int P, typename Real, int LAYOUT>
__device__ void warp_traverse(const SysDev& S, const TravPts& T, WarpStore& W, unsigned pmask,
                              int (*path)[BHMC_MAX_D + 1], TravOut& out) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  if (lane == 0) W.stk[0] = make_uint2(0u, pmask);
  int top = 1;
  __syncwarp();
  Acc<Real> acc;
  int visited = 0, accepted = 0, pairs = 0, fp64 = 0, err = 0;
  int cp = 1;
  while (cp < S.C) cp <<= 1;
  const int lg = 31 - __clz(cp);
  int rounds = 0;
  while (top > 0) {
    if (++rounds > (1 << 22)) {
      err = BHMC_ETIMEOUT;
      break;
    }
    const int npop = min(top, 4);
    const int g = lane >> 3;
    uint2 e = make_uint2(0u, 0u);
    if (g < npop) e = W.stk[top - 1 - g];
    __syncwarp();
    top -= npop;
    const int node = (int)e.x + (lane & 7);
    const unsigned om = e.y & 15u, fd = (e.y >> 4) & 15u;
    unsigned mac = 0, open = 0, fdc = 0, dir = 0;
    int fc = -1, cnt = 0;
    bool corr = false;
    if (g < npop && (om | fd)) {
      const int4 b = S.nB[node];
      const unsigned long long key = ((unsigned long long)(unsigned)b.w << 32) | (unsigned)b.z;
      if (key != 0ULL) {
        fc = b.x;
        cnt = b.y;
        const int d = key_depth(key);
        const int sh = 3 * (S.Dmax - d);
        int in_s = 0;
        for (int k = 0; k < T.n_excl; ++k) in_s += ((T.ekey[k] >> sh) == key) ? 1 : 0;
        if (path) {
          unsigned all = om | fd;
          while (all) {
            const int s = __ffs(all) - 1;
            all &= all - 1;
            if ((T.pkey[s] >> sh) == key) path[s][d] = node;
          }
        }
        visited += __popc(om);
        const int np = cnt - in_s;
        corr = in_s > 0;
        if (np > 0) {
          const float4 a = S.nA[node];
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
    }
    // children to the stack
    const bool push = (open | fdc) != 0;
    const unsigned pb = __ballot_sync(FULL, push);
    const int npush = __popc(pb);
    if (top + npush > BHMC_STACK) {
      err = BHMC_ESTACK;
      break;
    }
    if (push) W.stk[top + __popc(pb & lanemask_lt())] = make_uint2((unsigned)fc, open | (fdc << 4));
    top += npush;
    // multipole items
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
        W.mi[pos++] = ((unsigned)node << 3) | (corr ? 4u : 0u) | (unsigned)s;
      }
    }
    accepted += nm;
    // direct items
    const unsigned db = __ballot_sync(FULL, dir != 0);
    const int ndir = __popc(db);
    if (dir) W.di[__popc(db & lanemask_lt())] = make_uint2((unsigned)node, ((unsigned)cnt << 4) | dir);
    __syncwarp();
    for (int k = lane; k < total; k += 32) {
      const unsigned it = W.mi[k];
      const int s = (int)(it & 3u);
      const Real v = eval_item<P, Real, LAYOUT>(S, T, (int)(it >> 3), s, (it & 4u) != 0);
      acc.add(sizeof(Real) == 4 ? (Real)(T.w[s] * (float)v) : (Real)(T.w64[s] * (double)v));
    }
    const int per = 32 >> lg;
    for (int base = 0; base < ndir; base += per) {
      const int item = base + (lane >> lg);
      const int k = lane & (cp - 1);
      if (item < ndir) {
        const uint2 di = W.di[item];
        const int c = (int)(di.y >> 4);
        if (k < c) {
          const int slot = (int)di.x * (S.C + 2) + k;
          const float4 sa = S.sA[slot];
          const float4 sb = S.sB[slot];
          const int j = __float_as_int(sb.w);
          bool skip = false;
          for (int u = 0; u < T.n_excl; ++u) skip |= (T.excl[u] == j);
          if (!skip) {
            unsigned m = di.y & 15u;
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
        }
      }
    }
    __syncwarp();
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
