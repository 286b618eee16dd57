// bhmc_energy.cuh -- total treecode energy E = (1/2) l_B sum_j q_j phi_{T\{j}}(r_j)
// (Eq. 1.1 evaluated with the traversal of Sec. 3.2 for every charge).
//
// One warp evaluates 32 targets that are neighbours in Morton order.  The warp
// walks the union of their traversals: a stack entry is a group of eight
// sibling clusters with two 32-bit lane masks (lanes still traversing it, and
// lanes summing it directly after a MAC failure with N' <= N0).  Every lane
// takes its own MAC decision for its own target, so each target's interaction
// list is exactly the one of its own traversal; lanes that agree share the
// cluster loads (broadcast reads).
#pragma once

#include "bhmc_traverse.cuh"

#define BHMC_ESTACK_ENTRIES 512

namespace bhmc {

struct EnergyStack {
  int4 e[BHMC_ESTACK_ENTRIES];  // {first node of the group, open lanes, direct lanes, unused}
};

template <typename Real>
__device__ __forceinline__ bool lane_mac(const SysDev& S, const float4& a, const double x[3], const float hi[3],
                                         const float lo[3]) {
  if (sizeof(Real) == 4) {
    const float rx = (a.x - hi[0]) - lo[0], ry = (a.y - hi[1]) - lo[1], rz = (a.z - hi[2]) - lo[2];
    const float t = S.theta2f * (rx * rx + ry * ry + rz * rz);
    const float rho2 = 3.0f * a.w * a.w;
    if (t >= rho2 * 1.0000076293945312f) return true;
    if (t <= rho2 * 0.9999923706054688f) return false;
  }
  const double dx = __dsub_rn((double)a.x, x[0]);
  const double dy = __dsub_rn((double)a.y, x[1]);
  const double dz = __dsub_rn((double)a.z, x[2]);
  const double dd = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  const double r2 = __dmul_rn(__dmul_rn(3.0, (double)a.w), (double)a.w);
  return r2 <= __dmul_rn(S.theta2, dd);
}

template <int P, typename Real, int LAYOUT>
__device__ __forceinline__ Real lane_multipole(const SysDev& S, const float4& a, int node, const double x[3],
                                               const float hi[3], const float lo[3], bool self, double q,
                                               const float qhi[3], const float qlo[3]) {
  constexpr int K = nterms(P);
  if (sizeof(Real) == 4 && P < 6) {
    // the recurrence (measured faster than the coefficient form up to p = 4)
    const float rx = (a.x - hi[0]) - lo[0], ry = (a.y - hi[1]) - lo[1], rz = (a.z - hi[2]) - lo[2];
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
    if (self) {  // the target's own charge lies in the cluster: remove its expansion
      const float dx = (qhi[0] - a.x) + qlo[0], dy = (qhi[1] - a.y) + qlo[1], dz = (qhi[2] - a.z) + qlo[2];
      v -= (float)q * dot_monomials<P, float>(Tc, dx, dy, dz);
    }
    return (Real)v;
  }
  if (sizeof(Real) == 4) {
    // p >= 6: evaluation coefficients (a third of the recurrence's instructions)
    const float rx = (a.x - hi[0]) - lo[0], ry = (a.y - hi[1]) - lo[1], rz = (a.z - hi[2]) - lo[2];
    // the target's own charge, if it lies in the cluster, is removed through its expansion
    const float qe[1] = {(float)q};
    const float de[1][3] = {{(qhi[0] - a.x) + qlo[0], (qhi[1] - a.y) + qlo[1], (qhi[2] - a.z) + qlo[2]}};
    return (Real)w_multipole<P, LAYOUT>(S, node, rx, ry, rz, self ? 1 : 0, qe, de);
  } else {
    const double rx = __dsub_rn((double)a.x, x[0]), ry = __dsub_rn((double)a.y, x[1]),
                 rz = __dsub_rn((double)a.z, x[2]);
    double Tc[K];
    taylor<P, double>(rx, ry, rz, Tc);
    const double* M = S.M64 + (size_t)node * K;
    double v = 0.0;
#pragma unroll
    for (int t = 0; t < K; ++t) v += Tc[t] * M[t];
    if (self)
      v -= q * dot_monomials<P, double>(Tc, __dsub_rn(x[0], (double)a.x), __dsub_rn(x[1], (double)a.y),
                                         __dsub_rn(x[2], (double)a.z));
    return (Real)v;
  }
}

// partial[warp] = sum over the warp's targets of q_j phi_{T\{j}}(r_j); phi (may
// be null) receives every target's potential; cnt (may be null) accumulates the
// interaction-list counters {visited, multipole, direct pairs} over all targets.
template <int P, typename Real, int LAYOUT>
__global__ void __launch_bounds__(128) k_energy(SysDev S, const int* order, double* partial, double* phi,
                                                int* err, unsigned long long* cnt) {
  __shared__ EnergyStack stk[4];
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int warp = blockIdx.x * (blockDim.x >> 5) + wib;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  EnergyStack& E = stk[wib];
  const int SC = S.C + 2;
  double wsum = 0.0;
  int errv = 0;
  unsigned c_vis = 0, c_acc = 0, c_pairs = 0;
  for (int base = warp * 32; base < S.n_tree; base += nwarps * 32) {
    const int jj = base + lane;
    const bool valid = jj < S.n_tree;
    const int j = valid ? order[jj] : 0;
    double x[3] = {S.px[j], S.py[j], S.pz[j]};
    float hi[3], lo[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float2 f = split2(x[k]);
      hi[k] = f.x;
      lo[k] = f.y;
    }
    const double q = S.pq[j];
    const unsigned long long kj = S.ckey[j];
    Acc<Real> acc;
    const unsigned lanes = __ballot_sync(FULL, valid);
    if (lane == 0) E.e[0] = make_int4(0, (int)lanes, 0, 0);
    int top = 1;
    __syncwarp();
    int rounds = 0;
    while (top > 0) {
      if (++rounds > S.pass_pops) {
        errv = BHMC_ETIMEOUT;
        break;
      }
      const int4 en = E.e[--top];
      __syncwarp();
      // headers of the group's eight clusters: lane o loads cluster o
      const int4 hb = S.nB[en.x + (lane & 7)];
      const float4 ha = S.nA[en.x + (lane & 7)];
      const unsigned om = (unsigned)en.y, fm = (unsigned)en.z;
      const bool in_om = (om >> lane) & 1u, in_fm = (fm >> lane) & 1u;
#pragma unroll 1
      for (int o = 0; o < 8; ++o) {
        int4 b;
        b.x = __shfl_sync(FULL, hb.x, o);
        b.y = __shfl_sync(FULL, hb.y, o);
        b.z = __shfl_sync(FULL, hb.z, o);
        b.w = __shfl_sync(FULL, hb.w, o);
        float4 a;
        a.x = __shfl_sync(FULL, ha.x, o);
        a.y = __shfl_sync(FULL, ha.y, o);
        a.z = __shfl_sync(FULL, ha.z, o);
        a.w = __shfl_sync(FULL, ha.w, o);
        const unsigned long long key = ((unsigned long long)(unsigned)b.w << 32) | (unsigned)b.z;
        if (key == 0ULL) continue;  // empty slot of the root group
        c_vis += in_om ? 1u : 0u;
        if (b.y == 0) continue;     // empty cluster
        const int node = en.x + o;
        const int sh = 3 * (S.Dmax - key_depth(key));
        const bool self = (kj >> sh) == key;
        const int np = b.y - (self ? 1 : 0);
        bool mul = false, opn = false, fdv = false, dir = false;
        if (in_om && np > 0) {
          if (np >= S.N0 && lane_mac<Real>(S, a, x, hi, lo))
            mul = true;
          else if (b.x >= 0)
            (np > S.N0 ? opn : fdv) = true;
          else
            dir = true;
        }
        if (in_fm && np > 0) {
          if (b.x >= 0)
            fdv = true;
          else
            dir = true;
        }
        if (mul) {
          acc.add(lane_multipole<P, Real, LAYOUT>(S, a, node, x, hi, lo, self, q, hi, lo));
          ++c_acc;
        }
        const unsigned mo = __ballot_sync(FULL, opn), mf = __ballot_sync(FULL, fdv);
        if (mo | mf) {
          if (top >= BHMC_ESTACK_ENTRIES) {
            errv = BHMC_ESTACK;
            top = 0;
            break;
          }
          if (lane == 0) E.e[top] = make_int4(b.x, (int)mo, (int)mf, 0);
          ++top;
        }
        if (__any_sync(FULL, dir)) {
          for (int k = 0; k < b.y; ++k) {
            const float4 sa = S.sA[node * SC + k];
            const float4 sb = S.sB[node * SC + k];
            if (dir && __float_as_int(sb.w) != j) {
              ++c_pairs;
              if (sizeof(Real) == 4) {
                const float dx = (sa.x - hi[0]) + (sb.x - lo[0]);
                const float dy = (sa.y - hi[1]) + (sb.y - lo[1]);
                const float dz = (sa.z - hi[2]) + (sb.z - lo[2]);
                acc.add((Real)(sa.w * rsqrtf(dx * dx + dy * dy + dz * dz)));
              } else {
                const int jd = __float_as_int(sb.w);
                const double dx = S.px[jd] - x[0], dy = S.py[jd] - x[1], dz = S.pz[jd] - x[2];
                acc.add((Real)(S.pq[jd] / sqrt(dx * dx + dy * dy + dz * dz)));
              }
            }
          }
        }
      }
      __syncwarp();
    }
    if (valid) {
      wsum += q * acc.value();
      if (phi) phi[j] = acc.value();
    }
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(FULL, wsum, o);
  if (lane == 0) {
    partial[warp] = wsum;
    if (errv) atomicCAS(err, 0, errv);
  }
  if (cnt) {
    unsigned long long v0 = c_vis, v1 = c_acc, v2 = c_pairs;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v0 += __shfl_xor_sync(FULL, v0, o);
      v1 += __shfl_xor_sync(FULL, v1, o);
      v2 += __shfl_xor_sync(FULL, v2, o);
    }
    if (lane == 0) {
      atomicAdd(cnt, v0);
      atomicAdd(cnt + 1, v1);
      atomicAdd(cnt + 2, v2);
    }
  }
}

}  // namespace bhmc
