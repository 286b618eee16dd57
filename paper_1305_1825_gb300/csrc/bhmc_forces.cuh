// bhmc_forces.cuh -- adjoint of the total treecode energy: dE/dr_k and dE/dq_k
// of every charge with the MAC decisions held fixed.
//
// E = (1/2) l_B sum_i q_i phi_i, phi_i = sum_{A accepted} sum_n T_n(r_A - r_i) M_A^n
//                                       + sum_{j direct} q_j / |r_j - r_i|.
// Pass 1 (k_forces_traverse, the warp-union traversal of the energy kernel):
//   phi_i and the target gradient grad phi_i (d/dx T_n(r_A - x) =
//   -(n_c + 1) T_{n+e_c}); the cluster adjoints lambda_A^n += q_i T_n(r_A - r_i);
//   direct pairs' source terms psi_j += q_i/r and s_j += -q_i q_j (r_j - r_i)/r^3.
//   The warp's lanes reduce-scatter their contributions, so that each sum is
//   added by one FP64 atomic from the lane that holds it.
// Pass 2 (k_forces_push): every charge k walks the clusters containing it and
//   collects sum_n lambda_A^n (r_k - r_A)^n (for dE/dq_k) and
//   q_k sum_n lambda_A^n d/dr_k (r_k - r_A)^n (for dE/dr_k).
#pragma once

#include "bhmc_energy.cuh"

namespace bhmc {

// Sums over the 32 lanes of v[0..KP), scattered: afterwards lane L holds the
// sums of terms M L .. M L + M - 1 in v[0..M), M = KP / 32.  Recursive halving:
// at each of five steps a lane keeps half of its terms and adds its partner's
// values of them, KP - M shuffles in all (a butterfly per term takes 5 KP).
template <int KP, int N, typename R>
__device__ __forceinline__ void warp_reduce_scatter(R (&v)[N], int lane) {
  static_assert(KP % 32 == 0 && KP <= N, "KP must be a multiple of 32 within the array");
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const int o = 16 >> st, half = KP >> (st + 1);
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < half; ++j) {
      const R a = v[j], b = v[j + half];
      const R keep = up ? b : a, send = up ? a : b;
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
}

template <int P, typename Real, int LAYOUT>
__global__ void __launch_bounds__(128) k_forces_traverse(SysDev S, const int* order, double* phi_out,
                                                         double* tgrad, double* lam, double* psi, double* src,
                                                         int* err) {
  constexpr int K = nterms(P);
  constexpr int K1 = nterms(P + 1);
  constexpr int KP = (K + 31) / 32 * 32;            // adjoint terms padded for the reduce-scatter
  constexpr int NT = K1 > KP ? K1 : KP;
  __shared__ EnergyStack stk[4];
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int warp = blockIdx.x * (blockDim.x >> 5) + wib;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  EnergyStack& E = stk[wib];
  const int SC = S.C + 2;
  int errv = 0;
  for (int base = warp * 32; base < S.n_tree; base += nwarps * 32) {
    const int jj = base + lane;
    const bool valid = jj < S.n_tree;
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
      if (++rounds > S.pass_pops) {
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
          Real Tc[NT];
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
            taylor<P + 1, Real>(rx, ry, rz, *reinterpret_cast<Real(*)[K1]>(&Tc[0]));
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
              }
          if (mul) {
            phi.add(v);
            g0.add(d0);
            g1.add(d1);
            g2.add(d2);
          }
          // cluster adjoint: the warp's contributions q_i T_n summed in the
          // traversal precision (reduce-scatter), then one FP64 atomic per
          // term, issued by the lane that holds its sum
          const Real qm = mul ? (Real)qi : Real(0);
#pragma unroll
          for (int t = 0; t < KP; ++t) Tc[t] = t < K ? qm * Tc[t] : Real(0);
          warp_reduce_scatter<KP>(Tc, lane);
#pragma unroll
          for (int u = 0; u < KP / 32; ++u) {
            const int t = (KP / 32) * lane + u;
            if (t < K && Tc[u] != Real(0)) atomicAdd(&lam[(size_t)node * K + t], (double)Tc[u]);
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
          // eight slots at a time; their source terms (psi_j and the three
          // components of s_j) summed over the warp by one reduce-scatter,
          // after which lane 4u + c holds component c of slot u
          for (int k0 = 0; k0 < b.y; k0 += 8) {
            Real w[32];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              Real cp = 0, c0 = 0, c1 = 0, c2 = 0;
              const int k = k0 + u;
              if (k < b.y) {
                const float4 sa = S.sA[node * SC + k];
                const float4 sb = S.sB[node * SC + k];
                const int j = __float_as_int(sb.w);
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
              }
              w[4 * u + 0] = cp;
              w[4 * u + 1] = c0;
              w[4 * u + 2] = c1;
              w[4 * u + 3] = c2;
            }
            warp_reduce_scatter<32>(w, lane);
            const int u = lane >> 2, c = lane & 3;
            if (k0 + u < b.y && w[0] != Real(0)) {
              const int j = __float_as_int(S.sB[node * SC + k0 + u].w);
              atomicAdd(c == 0 ? &psi[j] : &src[3 * j + c - 1], (double)w[0]);
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
    // a fixed charge outside the tree belongs to no cluster
    for (int d = 0; d <= S.Dmax && !off_tree(S, k); ++d) {
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
