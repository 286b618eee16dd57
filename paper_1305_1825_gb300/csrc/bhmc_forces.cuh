// bhmc_forces.cuh -- adjoint of the total treecode energy: dE/dr_k and dE/dq_k
// of every charge with the MAC decisions held fixed.
//
// E = (1/2) l_B sum_i q_i phi_i, phi_i = sum_{A accepted} sum_n T_n(r_A - r_i) M_A^n
//                                       + sum_{j direct} q_j / |r_j - r_i|.
// Pass 1 (k_forces_traverse, the warp-union traversal of the energy kernel):
//   phi_i and the target gradient grad phi_i (d/dx T_n(r_A - x) =
//   -(n_c + 1) T_{n+e_c}); the cluster adjoints lambda_A^n += q_i T_n(r_A - r_i);
//   direct pairs' source terms psi_j += q_i/r and s_j += -q_i q_j (r_j - r_i)/r^3.
//   Lanes reduce their contributions to one value per warp before a single FP64
//   atomic add.
// Pass 2 (k_forces_push): every charge k walks the clusters containing it and
//   collects sum_n lambda_A^n (r_k - r_A)^n (for dE/dq_k) and
//   q_k sum_n lambda_A^n d/dr_k (r_k - r_A)^n (for dE/dr_k).
#pragma once

#include "bhmc_energy.cuh"

namespace bhmc {

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int P, typename Real, int LAYOUT>
__global__ void __launch_bounds__(128) k_forces_traverse(SysDev S, const int* order, double* phi_out,
                                                         double* tgrad, double* lam, double* psi, double* src,
                                                         int* err) {
  constexpr int K = nterms(P);
  constexpr int K1 = nterms(P + 1);
  __shared__ EnergyStack stk[4];
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int warp = blockIdx.x * (blockDim.x >> 5) + wib;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  EnergyStack& E = stk[wib];
  const int SC = S.C + 2;
  int errv = 0;
  for (int base = warp * 32; base < S.n_tot; base += nwarps * 32) {
    const int jj = base + lane;
    const bool valid = jj < S.n_tot;
    const int i = valid ? order[jj] : 0;
    const double x[3] = {S.px[i], S.py[i], S.pz[i]};
    float hi[3], lo[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float2 f = split2(x[k]);
      hi[k] = f.x;
      lo[k] = f.y;
    }
    const double qi = S.pq[i];
    const unsigned long long ki = S.ckey[i];
    // per-lane sums in the traversal precision (compensated in FP32)
    Acc<Real> phi, g0, g1, g2;
    const unsigned lanes = __ballot_sync(FULL, valid);
    if (lane == 0) E.e[0] = make_int4(0, (int)lanes, 0, 0);
    int top = 1;
    __syncwarp();
    int rounds = 0;
    while (top > 0) {
      if (++rounds > (1 << 24)) {
        errv = BHMC_ETIMEOUT;
        break;
      }
      const int4 en = E.e[--top];
      __syncwarp();
      const int4 hb = S.nB[en.x + (lane & 7)];
      const float4 ha = S.nA[en.x + (lane & 7)];
      const bool in_om = (((unsigned)en.y) >> lane) & 1u, in_fm = (((unsigned)en.z) >> lane) & 1u;
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
        if (key == 0ULL || b.y == 0) continue;
        const int node = en.x + o;
        const int sh = 3 * (S.Dmax - key_depth(key));
        const bool self = (ki >> sh) == key;
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
        if (__any_sync(FULL, mul)) {
          // Taylor coefficients to order p + 1 at R = r_A - x (an accepted cluster
          // never holds its own target, so M' = M)
          Real Tc[K1];
          {
            Real rx, ry, rz;
            if (sizeof(Real) == 4) {
              rx = (Real)((a.x - hi[0]) - lo[0]);
              ry = (Real)((a.y - hi[1]) - lo[1]);
              rz = (Real)((a.z - hi[2]) - lo[2]);
            } else {
              rx = (Real)__dsub_rn((double)a.x, x[0]);
              ry = (Real)__dsub_rn((double)a.y, x[1]);
              rz = (Real)__dsub_rn((double)a.z, x[2]);
            }
            taylor<P + 1, Real>(rx, ry, rz, Tc);
          }
          Real v = 0, d0 = 0, d1 = 0, d2 = 0;
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
                  m = (Real)(LAYOUT == BHMC_LAYOUT_AOS ? S.M32[(size_t)node * pad4(K) + t]
                                                       : S.M32[(size_t)t * S.node_cap + node]);
                else
                  m = (Real)S.M64[(size_t)node * K + t];
                v += Tc[t] * m;
                d0 -= Real(n1 + 1) * Tc[tidx(n1 + 1, n2, n3)] * m;
                d1 -= Real(n2 + 1) * Tc[tidx(n1, n2 + 1, n3)] * m;
                d2 -= Real(n3 + 1) * Tc[tidx(n1, n2, n3 + 1)] * m;
                // cluster adjoint: the warp's contributions summed in the
                // traversal precision, one FP64 atomic per term and warp
                const Real l = warp_sum<Real>(mul ? (Real)qi * Tc[t] : Real(0));
                if (lane == 0) atomicAdd(&lam[(size_t)node * K + t], (double)l);
              }
          if (mul) {
            phi.add(v);
            g0.add(d0);
            g1.add(d1);
            g2.add(d2);
          }
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
            const int j = __float_as_int(sb.w);
            Real cp = 0, c0 = 0, c1 = 0, c2 = 0;
            if (dir && j != i) {
              Real ex, ey, ez, qj;
              if (sizeof(Real) == 4) {
                ex = (Real)((sa.x - hi[0]) + (sb.x - lo[0]));
                ey = (Real)((sa.y - hi[1]) + (sb.y - lo[1]));
                ez = (Real)((sa.z - hi[2]) + (sb.z - lo[2]));
                qj = (Real)sa.w;
              } else {
                ex = (Real)(S.px[j] - x[0]);
                ey = (Real)(S.py[j] - x[1]);
                ez = (Real)(S.pz[j] - x[2]);
                qj = (Real)S.pq[j];
              }
              const Real r2 = ex * ex + ey * ey + ez * ez;
              const Real rinv = rsqrt_t<Real>(r2);
              const Real r3inv = rinv * rinv * rinv;
              phi.add(qj * rinv);
              g0.add(qj * ex * r3inv);
              g1.add(qj * ey * r3inv);
              g2.add(qj * ez * r3inv);
              const Real qr = (Real)qi;
              cp = qr * rinv;
              c0 = -qr * qj * ex * r3inv;
              c1 = -qr * qj * ey * r3inv;
              c2 = -qr * qj * ez * r3inv;
            }
            cp = warp_sum<Real>(cp);
            c0 = warp_sum<Real>(c0);
            c1 = warp_sum<Real>(c1);
            c2 = warp_sum<Real>(c2);
            if (lane == 0 && (cp != Real(0) || c0 != Real(0) || c1 != Real(0) || c2 != Real(0))) {
              atomicAdd(&psi[j], (double)cp);
              atomicAdd(&src[3 * j + 0], (double)c0);
              atomicAdd(&src[3 * j + 1], (double)c1);
              atomicAdd(&src[3 * j + 2], (double)c2);
            }
          }
        }
      }
      __syncwarp();
    }
    if (valid) {
      phi_out[i] = phi.value();
      tgrad[3 * i + 0] = qi * g0.value();
      tgrad[3 * i + 1] = qi * g1.value();
      tgrad[3 * i + 2] = qi * g2.value();
    }
    __syncwarp();
  }
  if (lane == 0 && errv) atomicCAS(err, 0, errv);
}

// Pass 2: one thread per charge, clusters from the root down to its leaf.
static __global__ void k_forces_push(SysDev S, const double* phi, const double* tgrad, const double* lam,
                              const double* psi, const double* src, double* dEdr, double* dEdq) {
  const double half = 0.5 * S.lB;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < S.n_tot; k += gridDim.x * blockDim.x) {
    const double x[3] = {S.px[k], S.py[k], S.pz[k]};
    const unsigned long long key = S.ckey[k];
    double gq = 0.0, gr0 = 0.0, gr1 = 0.0, gr2 = 0.0;
    int node = 0;
    for (int d = 0; d <= S.Dmax; ++d) {
      const float4 c = S.nA[node];
      const double r[3] = {x[0] - (double)c.x, x[1] - (double)c.y, x[2] - (double)c.z};
      double px[BHMC_MAX_P + 1], py[BHMC_MAX_P + 1], pz[BHMC_MAX_P + 1];
      px[0] = py[0] = pz[0] = 1.0;
      for (int e = 1; e <= S.p; ++e) {
        px[e] = px[e - 1] * r[0];
        py[e] = py[e - 1] * r[1];
        pz[e] = pz[e - 1] * r[2];
      }
      const double* L = lam + (size_t)node * S.K;
      int t = 0;
      for (int kk = 0; kk <= S.p; ++kk)
        for (int n1 = kk; n1 >= 0; --n1)
          for (int n2 = kk - n1; n2 >= 0; --n2, ++t) {
            const int n3 = kk - n1 - n2;
            const double l = L[t];
            gq += l * px[n1] * py[n2] * pz[n3];
            if (n1) gr0 += l * n1 * px[n1 - 1] * py[n2] * pz[n3];
            if (n2) gr1 += l * n2 * px[n1] * py[n2 - 1] * pz[n3];
            if (n3) gr2 += l * n3 * px[n1] * py[n2] * pz[n3 - 1];
          }
      const int fc = S.nB[node].x;
      if (fc < 0 || d >= S.Dmax) break;
      node = fc + (int)((key >> (3 * (S.Dmax - d - 1))) & 7ULL);
    }
    const double q = S.pq[k];
    dEdq[k] = half * (phi[k] + psi[k] + gq);
    dEdr[3 * k + 0] = half * (tgrad[3 * k + 0] + src[3 * k + 0] + q * gr0);
    dEdr[3 * k + 1] = half * (tgrad[3 * k + 1] + src[3 * k + 1] + q * gr1);
    dEdr[3 * k + 2] = half * (tgrad[3 * k + 2] + src[3 * k + 2] + q * gr2);
  }
}

}  // namespace bhmc
