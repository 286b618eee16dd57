// bhmc_traverse.cuh -- building blocks of the octree traversal (Sec. 3.2):
// the evaluation points, the MAC, the multipole term of a cluster with the
// excluded charges removed, direct leaf terms and compensated accumulation.
//
// The MAC decision of every (cluster, point) pair is the FP64 decision
// rho_A^2 <= theta^2 ((dx*dx + dy*dy) + dz*dz): FP32 settles it when the value
// is further than 2^-17 (relative) from the threshold, the exact FP64 sequence
// otherwise.  Error analysis: with x = hi + lo (hi = fl(x), lo = fl(x - hi)) and
// an exact FP32 centre c, R = (c - hi) - lo has |R - (c - x)| <= 2u|c - x| +
// 2u^2|x| (u = 2^-24); theta^2 |R|^2 in FP32 is then within about 10u relative of
// the exact value, well inside the 2^-17 band.
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

struct TravOut {
  double sum;
  int overlap;    // the trial point (point 1) lies within the hard core of a mobile ion
  // gradient traversals: potential and its gradient per role, role 0 the
  // points 0 and 1 (ion), role 1 the points 2 and 3 (image); a traversal
  // evaluates at most one point of each role
  double phi[2];
  double grad[2][3];
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

// Value and gradient with respect to the evaluation point of the p-th order
// expansion of one charge at offset d from the cluster centre, from Taylor
// coefficients up to order p + 1: d/dx T_n(r_A - x) = -(n_c + 1) T_{n + e_c}.
template <int P, typename R>
__device__ __forceinline__ void dot_monomials_grad(const R (&T)[nterms(P + 1)], R dx, R dy, R dz, R& v,
                                                   R& g0, R& g1, R& g2) {
  R px[P + 1], py[P + 1], pz[P + 1];
  px[0] = py[0] = pz[0] = R(1);
#pragma unroll
  for (int k = 1; k <= P; ++k) {
    px[k] = px[k - 1] * dx;
    py[k] = py[k - 1] * dy;
    pz[k] = pz[k - 1] * dz;
  }
  v = g0 = g1 = g2 = R(0);
#pragma unroll
  for (int k = 0; k <= P; ++k)
#pragma unroll
    for (int n1 = k; n1 >= 0; --n1)
#pragma unroll
      for (int n2 = k - n1; n2 >= 0; --n2) {
        const int n3 = k - n1 - n2;
        const R m = px[n1] * py[n2] * pz[n3];
        v += T[tidx(n1, n2, n3)] * m;
        g0 -= R(n1 + 1) * T[tidx(n1 + 1, n2, n3)] * m;
        g1 -= R(n2 + 1) * T[tidx(n1, n2 + 1, n3)] * m;
        g2 -= R(n3 + 1) * T[tidx(n1, n2, n3 + 1)] * m;
      }
}

// Multipole term of cluster `node` at point s and its gradient with respect to
// the evaluation point (excluded charges removed as in eval_item).
template <int P, typename Real, int LAYOUT>
__device__ __forceinline__ void eval_item_grad(const SysDev& S, const TravPts& T, int node, int s, unsigned emask,
                                               Real& v, Real& g0, Real& g1, Real& g2) {
  constexpr int K = nterms(P);
  const float4 a = S.nA[node];
  Real rx, ry, rz;
  if (sizeof(Real) == 4) {
    rx = (Real)((a.x - T.hi[s][0]) - T.lo[s][0]);
    ry = (Real)((a.y - T.hi[s][1]) - T.lo[s][1]);
    rz = (Real)((a.z - T.hi[s][2]) - T.lo[s][2]);
  } else {
    rx = (Real)__dsub_rn((double)a.x, T.x[s][0]);
    ry = (Real)__dsub_rn((double)a.y, T.x[s][1]);
    rz = (Real)__dsub_rn((double)a.z, T.x[s][2]);
  }
  Real Tc[nterms(P + 1)];
  taylor<P + 1, Real>(rx, ry, rz, Tc);
  v = g0 = g1 = g2 = Real(0);
#pragma unroll
  for (int k = 0; k <= P; ++k)
#pragma unroll
    for (int n1 = k; n1 >= 0; --n1)
#pragma unroll
      for (int n2 = k - n1; n2 >= 0; --n2) {
        const int n3 = k - n1 - n2;
        const int t = tidx(n1, n2, n3);
        Real m;
        if (sizeof(Real) == 4)
          m = (Real)(LAYOUT == BHMC_LAYOUT_AOS ? S.M32[(size_t)node * pad4(K) + t] : S.M32[(size_t)t * S.node_cap + node]);
        else
          m = (Real)S.M64[(size_t)node * K + t];
        v += Tc[t] * m;
        g0 -= Real(n1 + 1) * Tc[tidx(n1 + 1, n2, n3)] * m;
        g1 -= Real(n2 + 1) * Tc[tidx(n1, n2 + 1, n3)] * m;
        g2 -= Real(n3 + 1) * Tc[tidx(n1, n2, n3 + 1)] * m;
      }
  while (emask) {
    const int k = __ffs(emask) - 1;
    emask &= emask - 1;
    Real dx, dy, dz;
    if (sizeof(Real) == 4) {
      dx = (Real)((T.ehi[k][0] - a.x) + T.elo[k][0]);
      dy = (Real)((T.ehi[k][1] - a.y) + T.elo[k][1]);
      dz = (Real)((T.ehi[k][2] - a.z) + T.elo[k][2]);
    } else {
      dx = (Real)__dsub_rn(T.ex[k][0], (double)a.x);
      dy = (Real)__dsub_rn(T.ex[k][1], (double)a.y);
      dz = (Real)__dsub_rn(T.ex[k][2], (double)a.z);
    }
    Real cv, c0, c1, c2;
    dot_monomials_grad<P, Real>(Tc, dx, dy, dz, cv, c0, c1, c2);
    const Real qe = sizeof(Real) == 4 ? (Real)T.eqf[k] : (Real)T.eq[k];
    v -= qe * cv;
    g0 -= qe * c0;
    g1 -= qe * c1;
    g2 -= qe * c2;
  }
}

// FP32 multipole sum_{|n| <= p} T_n(R) M_n of cluster `node` from its
// evaluation coefficients: with u = R / r, sum_{|n| = k} T_n(R) M_n =
// r^-(k+1) sum_{|m| = k} W_m u^m, so the sum is r^-1 (P_0 + r^-1 (P_1 + ...)).
// Each of the `ne` charges (qe, offset d from the cluster centre) is removed
// through its own truncated expansion, sum_{|n| = k} T_n(R) d^n =
// (-1)^k Q_k r^-(k+1) with Q_0 = 1, Q_1 = u.d, Q_{k+1} = ((2k+1)(u.d) Q_k -
// k |d|^2 Q_{k-1}) / (k+1) (the Legendre recurrence; 1/|R + d| = sum_k
// (-1)^k |d|^k P_k(cos) / r^(k+1)).
template <int P, int LAYOUT>
__device__ __forceinline__ float w_multipole(const SysDev& S, int node, float rx, float ry, float rz, int ne,
                                             const float* qe, const float (*de)[3]) {
  constexpr int K = nterms(P), KP = pad4(K);
  float W[KP];
  if (LAYOUT == BHMC_LAYOUT_AOS) {
    const float4* W4 = reinterpret_cast<const float4*>(S.W32 + (size_t)node * KP);
#pragma unroll
    for (int t4 = 0; t4 < KP / 4; ++t4) {
      const float4 v = W4[t4];
      W[4 * t4] = v.x;
      W[4 * t4 + 1] = v.y;
      W[4 * t4 + 2] = v.z;
      W[4 * t4 + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int t = 0; t < K; ++t) W[t] = S.W32[(size_t)t * S.node_cap + node];
  }
  const float rinv = rsqrtf(rx * rx + ry * ry + rz * rz);
  const float ux = rx * rinv, uy = ry * rinv, uz = rz * rinv;
  float px[P + 1], py[P + 1], pz[P + 1];
  px[0] = py[0] = pz[0] = 1.f;
#pragma unroll
  for (int k = 1; k <= P; ++k) {
    px[k] = px[k - 1] * ux;
    py[k] = py[k - 1] * uy;
    pz[k] = pz[k - 1] * uz;
  }
  float pk[P + 1];
#pragma unroll
  for (int k = 0; k <= P; ++k) {
    float acc = 0.f;
#pragma unroll
    for (int n1 = k; n1 >= 0; --n1) {
      const float pxy0 = px[n1];
#pragma unroll
      for (int n2 = k - n1; n2 >= 0; --n2) {
        const int n3 = k - n1 - n2;
        acc = fmaf(W[tidx(n1, n2, n3)], (pxy0 * py[n2]) * pz[n3], acc);
      }
    }
    pk[k] = acc;
  }
  for (int e = 0; e < ne; ++e) {
    const float dx = de[e][0], dy = de[e][1], dz = de[e][2];
    const float sd = ux * dx + uy * dy + uz * dz, td = dx * dx + dy * dy + dz * dz;
    float q0 = 1.f, q1 = sd;
    pk[0] -= qe[e];
    if constexpr (P >= 1) pk[1] += qe[e] * q1;
#pragma unroll
    for (int k = 1; k < P; ++k) {
      const float q2 = ((2.f * k + 1.f) * sd * q1 - (float)k * td * q0) * (1.f / (k + 1.f));
      pk[k + 1] += ((k + 1) & 1) ? qe[e] * q2 : -qe[e] * q2;
      q0 = q1;
      q1 = q2;
    }
  }
  float acc = pk[P];
#pragma unroll
  for (int k = P - 1; k >= 0; --k) acc = fmaf(acc, rinv, pk[k]);
  return acc * rinv;
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
  __device__ __forceinline__ void pair(float& h, float& l) const {  // value = h + l
    h = s;
    l = -c;
  }
};
template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double value() const { return s; }
};

// Potential and gradient sums of the two roles of a gradient traversal.
template <typename Real>
struct GradAcc {
  Acc<Real> phi[2];
  Real g[2][3] = {{Real(0), Real(0), Real(0)}, {Real(0), Real(0), Real(0)}};
  __device__ __forceinline__ void add(int s, Real v, Real gx, Real gy, Real gz) {
    if (s & 2) {
      phi[1].add(v);
      g[1][0] += gx;
      g[1][1] += gy;
      g[1][2] += gz;
    } else {
      phi[0].add(v);
      g[0][0] += gx;
      g[0][1] += gy;
      g[0][2] += gz;
    }
  }
};

// Direct terms of one leaf slot against the points of `m`, with gradients
// d/dx q_j/|r_j - x| = q_j (r_j - x)/|r_j - x|^3.
template <typename Real>
__device__ __forceinline__ void direct_slot_grad(const SysDev& S, const TravPts& T, float4 sa, float4 sb,
                                                 unsigned m, GradAcc<Real>& G, int& pairs) {
  const int j = __float_as_int(sb.w);
  for (int u = 0; u < T.n_excl; ++u)
    if (T.excl[u] == j) return;
  while (m) {
    const int s = __ffs(m) - 1;
    m &= m - 1;
    Real dx, dy, dz, qj;
    if (sizeof(Real) == 4) {
      dx = (Real)((sa.x - T.hi[s][0]) + (sb.x - T.lo[s][0]));
      dy = (Real)((sa.y - T.hi[s][1]) + (sb.y - T.lo[s][1]));
      dz = (Real)((sa.z - T.hi[s][2]) + (sb.z - T.lo[s][2]));
      qj = (Real)sa.w;
    } else {
      dx = (Real)__dsub_rn(S.px[j], T.x[s][0]);
      dy = (Real)__dsub_rn(S.py[j], T.x[s][1]);
      dz = (Real)__dsub_rn(S.pz[j], T.x[s][2]);
      qj = (Real)S.pq[j];
    }
    const Real r2 = dx * dx + dy * dy + dz * dz;
    const Real rinv = sizeof(Real) == 4 ? (Real)rsqrtf((float)r2) : (Real)(1.0 / sqrt((double)r2));
    const Real v = qj * rinv, f = v * rinv * rinv;
    G.add(s, v, f * dx, f * dy, f * dz);
    ++pairs;
  }
}

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

// Hard core of Eq. (2.1) at the trial position (point 1): the slot's charge,
// if a mobile ion other than the moved one, lies within the diameter.  FP32
// float-pair distances settle it outside a 2^-16 band around the contact
// distance; inside the band, the FP64 test of the definition.
__device__ __forceinline__ bool hc_slot(const SysDev& S, const TravPts& T, float4 sa, float4 sb) {
  const int j = __float_as_int(sb.w);
  if (j >= S.n_mob || j == T.excl[0]) return false;
  const float dx = (sa.x - T.hi[1][0]) + (sb.x - T.lo[1][0]);
  const float dy = (sa.y - T.hi[1][1]) + (sb.y - T.lo[1][1]);
  const float dz = (sa.z - T.hi[1][2]) + (sb.z - T.lo[1][2]);
  const float r2 = dx * dx + dy * dy + dz * dz;
  if (r2 > S.hc2f * 1.0000153f) return false;
  if (r2 < S.hc2f * 0.9999847f) return true;
  const double ex = __dsub_rn(T.x[1][0], S.px[j]), ey = __dsub_rn(T.x[1][1], S.py[j]);
  const double ez = __dsub_rn(T.x[1][2], S.pz[j]);
  return __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)) <= S.hc2;
}

// Whether the cluster box {centre, h} comes within the hard-core diameter of
// point 1 (conservative: a box that does is never reported as out of reach).
__device__ __forceinline__ bool hc_box(const SysDev& S, const TravPts& T, float4 a) {
  const float4 h = T.h4[1], l = T.l4[1];
  const float ex = fmaxf(fabsf((a.x - h.x) - l.x) - a.w, 0.f);
  const float ey = fmaxf(fabsf((a.y - h.y) - l.y) - a.w, 0.f);
  const float ez = fmaxf(fabsf((a.z - h.z) - l.z) - a.w, 0.f);
  return ex * ex + ey * ey + ez * ez <= S.hc2f * 1.001f;
}

}  // namespace bhmc
