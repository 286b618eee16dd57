// bhmc_block.cuh -- block-cooperative octree traversal for one trial move.
//
// All warps of the block share one frontier: a round pops up to blockDim/8
// groups of eight sibling clusters (one cluster per thread) from a stack in
// shared memory, classifies every (cluster, point) pair with the MAC of
// Sec. 3.2, pushes the groups to open, and evaluates the round's multipole and
// direct terms with all threads.  The four evaluation points of a move (ion
// and image, old and new positions) travel together as a 4-bit mask, so a
// cluster needed by several points is read once.  The headers of the next
// round are loaded before the current round's terms are evaluated.
#pragma once

#include "bhmc_traverse.cuh"

#define BHMC_BSTACK 4096
#define BHMC_PCNT_LEAF (1 << 30)  // path count entry of a leaf (never merged)
#define BHMC_PCNT_NONE (-1)       // path count entry not yet read

namespace bhmc {

// Loads issued at a fixed point of the instruction stream (the traversal
// pipelines them one round ahead) and L2 prefetches of whole lines.
__device__ __forceinline__ int4 ld_int4(const int4* p) {
  int4 v;
  asm volatile("ld.global.v4.s32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ float4 ld_float4(const float4* p) {
  float4 v;
  asm volatile("ld.global.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Lines of [p, p + bytes) into L1.
__device__ __forceinline__ void prefetch_range(const void* p, int bytes) {
  const char* c = reinterpret_cast<const char*>(p);
  for (int o = 0; o < bytes; o += 128) prefetch_l1(c + o);
  prefetch_l1(c + bytes - 1);
}

struct BlockStore {
  uint2 stk[BHMC_BSTACK];
  unsigned mi[4 * 32 * BHMC_MAX_WARPS];  // node << 4 | excluded mask << 2 | point
  uint2 di[32 * BHMC_MAX_WARPS];         // {leaf, count << 4 | point mask}
  int wcnt[BHMC_MAX_WARPS][3];
  double wsum[BHMC_MAX_WARPS];
  float wsf[BHMC_MAX_WARPS][2];
  int wred[BHMC_MAX_WARPS][6];
  double wg[BHMC_MAX_WARPS][8];
};

// h + l += h2 + l2 for unevaluated pairs of floats (Knuth's two-sum of the
// high parts, the low parts carried): about 44 significant bits, from FP32
// arithmetic alone.
__device__ __forceinline__ void df_add(float& h, float& l, float h2, float l2) {
  const float s = __fadd_rn(h, h2);
  const float bb = __fsub_rn(s, h);
  const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(h2, bb));
  const float t = __fadd_rn(e, __fadd_rn(l, l2));
  h = __fadd_rn(s, t);
  l = __fsub_rn(t, __fsub_rn(h, s));
}

// `path` (may be null) receives per point and level the cluster containing the
// point, `pcnt` (with path) that cluster's charge count when internal and
// BHMC_PCNT_LEAF for a leaf; `leafcnt[s]` the count of point s's leaf when the
// traversal reaches it.
// GRAD: instead of the weighted sum, accumulate the potential and its
// gradient per role (ion point, image point).
template <int P, typename Real, int LAYOUT, bool GRAD = false>
__device__ void block_traverse(const SysDev& S, const TravPts& T, BlockStore& B, unsigned pmask,
                               int (*path)[BHMC_MAX_D + 1], int (*pcnt)[BHMC_MAX_D + 1], int* leafcnt,
                               TravOut& out) {
  const unsigned FULL = 0xffffffffu;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nth = blockDim.x, NW = nth >> 5, G = nth >> 3;
  const int g = tid >> 3;
  const unsigned lt = lanemask_lt();
  Acc<Real> acc;
  GradAcc<Real> ga;
  int visited = 0, accepted = 0, pairs = 0, fp64 = 0, err = 0;
  const bool hc = S.hc2 > 0.0;  // hard cores (Eq. 2.1) at the trial point
  bool ovl = false;
  int cp = 1;
  while (cp < S.C) cp <<= 1;
  const int lg = 31 - __clz(cp);
  const int SC = S.C + 2;
  int top = 0, npop = 1;
  // A stack entry is a group of eight sibling clusters: {first node, bits 0-3
  // points still traversing, bits 4-7 points summing directly, bits 8-11
  // points whose own cluster is the group's parent, bits 12-16 depth, bit 17
  // reached only for the hard-core test of the trial point}.
  unsigned pm0 = 0;
#pragma unroll
  for (int s = 0; s < 4; ++s) pm0 |= T.pkey[s] != 0ULL ? (1u << s) : 0u;
  // Every point lies in the root cube, so the root fails the MAC (rho^2 =
  // 3h^2 > theta^2 d^2 for theta < 1); when it is internal with N' > N0 the
  // walk starts from its children, and the root counts as visited.
  const int4 rb = ld_int4(S.nB);
  const bool skip_root = rb.x >= 0 && rb.y - T.n_excl > S.N0;
  const int g0 = skip_root ? rb.x : 0;
  uint2 e = make_uint2((unsigned)g0, g == 0 ? (pmask | (pm0 << 8) | (skip_root ? (1u << 12) : 0u)) : 0u);
  if (skip_root && tid == 0) {
    visited += __popc(pmask);
    if (path)
      for (int s = 0; s < 4; ++s)
        if ((pmask >> s) & 1u) {
          path[s][0] = 0;
          pcnt[s][0] = rb.y;
        }
  }
  int4 b = make_int4(-1, 0, 0, 0);
  float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
  if (g == 0) {
    b = ld_int4(S.nB + g0 + (tid & 7));
    a = ld_float4(S.nA + g0 + (tid & 7));
  }
  // Multipole and direct terms of one round's item lists; the first direct
  // pass's slot loads are issued before the multipole work.
  auto run_items = [&](int tm_, int td_) {
    const int per = nth >> lg;
    // multipole items go from the top thread down and direct lanes from the
    // bottom up: the threads that take a busy round's second multipole item
    // get no direct term and, when the next round pops fewer groups than the
    // block has, no cluster to classify either
    const int kk = tid & (cp - 1);
    uint2 di0 = make_uint2(0u, 0u);
    float4 sa0 = make_float4(0.f, 0.f, 0.f, 0.f), sb0 = sa0;
    bool have0 = false;
    if ((tid >> lg) < td_) {
      di0 = B.di[tid >> lg];
      if (kk < (int)((di0.y >> 4) & 0xffffu)) {
        const int slot = (int)di0.x * SC + kk;
        sa0 = S.sA[slot];
        sb0 = S.sB[slot];
        have0 = true;
      }
    }
    for (int k = nth - 1 - tid; k < tm_; k += nth) {
      const unsigned it = B.mi[k];
      const int s = (int)(it & 3u);
      if (GRAD) {
        Real v, g0, g1, g2;
        eval_item_grad<P, Real, LAYOUT>(S, T, (int)(it >> 4), s, (it >> 2) & 3u, v, g0, g1, g2);
        ga.add(s, v, g0, g1, g2);
      } else {
        const Real v = eval_item<P, Real, LAYOUT>(S, T, (int)(it >> 4), s, (it >> 2) & 3u);
        acc.add(sizeof(Real) == 4 ? (Real)(T.w[s] * (float)v) : (Real)(T.w64[s] * (double)v));
      }
    }
    if (have0) {
      if (GRAD)
        direct_slot_grad<Real>(S, T, sa0, sb0, di0.y & 15u, ga, pairs);
      else
        direct_slot<Real>(S, T, sa0, sb0, di0.y & 15u, acc, pairs);
      if (hc && ((di0.y & 2u) || (di0.y >> 30))) ovl |= hc_slot(S, T, sa0, sb0);
    }
    for (int base = per; base < td_; base += per) {
      const int item = base + (tid >> lg);
      if (item < td_) {
        const uint2 di = B.di[item];
        if (kk < (int)((di.y >> 4) & 0xffffu)) {
          const int slot = (int)di.x * SC + kk;
          const float4 sa = S.sA[slot], sb = S.sB[slot];
          if (GRAD)
            direct_slot_grad<Real>(S, T, sa, sb, di.y & 15u, ga, pairs);
          else
            direct_slot<Real>(S, T, sa, sb, di.y & 15u, acc, pairs);
          if (hc && ((di.y & 2u) || (di.y >> 30))) ovl |= hc_slot(S, T, sa, sb);
        }
      }
    }
  };
  int rounds = 0;
  while (npop > 0) {
    if (++rounds > S.move_rounds) {
      err = BHMC_ETIMEOUT;
      break;
    }
    const int node = (int)e.x + (tid & 7);
    const unsigned om = e.y & 15u, fd = (e.y >> 4) & 15u, pmp = (e.y >> 8) & 15u;
    const int d = (int)((e.y >> 12) & 31u);
    const bool ovin = ((e.y >> 17) & 1u) != 0u;
    bool ovp = false, ovd = false;  // hard-core descent / leaf test for the trial point
    unsigned mac = 0, open = 0, fdc = 0, dir = 0, emask = 0, onp = 0;
    int fc = -1, cnt = 0;
    const unsigned long long key = ((unsigned long long)(unsigned)b.w << 32) | (unsigned)b.z;
    if (g < npop && ((om | fd) || ovin) && key != 0ULL) {
      fc = b.x;
      cnt = b.y;
      // points inside this cluster: those inside the parent whose octant at
      // this depth is this cluster's (the root holds every point in the cube)
      if (pmp) {
        if (d == 0) {
          onp = pmp;
        } else {
          const int sh = 3 * (S.Dmax - d);
          const unsigned o = (unsigned)(tid & 7);
#pragma unroll
          for (int s = 0; s < 4; ++s)
            if (((pmp >> s) & 1u) && (unsigned)((T.pkey[s] >> sh) & 7ULL) == o) onp |= 1u << s;
        }
      }
      // the excluded charges are the ion and its image at points 0 and 2
      emask = (onp & 1u) | (T.n_excl > 1 ? ((onp >> 1) & 2u) : 0u);
      if (path) {
        unsigned pr = onp & (om | fd);
        while (pr) {
          const int s = __ffs(pr) - 1;
          pr &= pr - 1;
          path[s][d] = node;
          pcnt[s][d] = fc >= 0 ? cnt : BHMC_PCNT_LEAF;
          if (fc < 0) leafcnt[s] = cnt;
        }
      }
      visited += __popc(om);
      const int np = cnt - __popc(emask);
      if (np > 0) {
        // MAC for the four points at once (independent chains, predicated)
        unsigned acc4 = 0, amb4 = 0;
        if (sizeof(Real) == 4) {
          const float rho2 = 3.0f * a.w * a.w;
          const float hi_t = rho2 * 1.0000076293945312f, lo_t = rho2 * 0.9999923706054688f;
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            const float4 h = T.h4[s], l = T.l4[s];
            const float rx = (a.x - h.x) - l.x, ry = (a.y - h.y) - l.y, rz = (a.z - h.z) - l.z;
            const float tt = S.theta2f * (rx * rx + ry * ry + rz * rz);
            acc4 |= (tt >= hi_t) ? (1u << s) : 0u;
            amb4 |= (tt > lo_t && tt < hi_t) ? (1u << s) : 0u;
          }
          amb4 &= om;
          while (amb4) {  // within 2^-17 of the threshold: exact FP64 decision
            const int s = __ffs(amb4) - 1;
            amb4 &= amb4 - 1;
            if (mac_test<double>(S, a, T, s, fp64)) acc4 |= 1u << s;
            ++fp64;
          }
        } else {
          unsigned m = om;
          while (m) {
            const int s = __ffs(m) - 1;
            m &= m - 1;
            if (mac_test<double>(S, a, T, s, fp64)) acc4 |= 1u << s;
          }
        }
        const unsigned ok = (np >= S.N0) ? acc4 & om : 0u;
        const unsigned rest = om & ~ok;
        mac = ok;
        if (fc >= 0) {
          if (np > S.N0)
            open = rest;
          else
            fdc = rest;
          fdc |= fd;
        } else {
          dir = rest | fd;
        }
        // hard core: a cluster the trial point accepted (or reached for this
        // test only) may still hold ions within the diameter of it
        if (hc && (ovin || (mac & 2u)) && hc_box(S, T, a)) {
          if (fc >= 0)
            ovp = true;
          else
            ovd = true;
        }
        if (LAYOUT == BHMC_LAYOUT_AOS && mac)
          prefetch_range(S.M32 + (size_t)node * pad4(nterms(P)), pad4(nterms(P)) * 4);
        if ((open | fdc) && fc >= 0) {  // the children's headers, popped next round
          prefetch_l1(S.nA + fc);
          prefetch_l1(S.nB + fc);
        }
        if (dir || ovd) {
          prefetch_range(S.sA + (size_t)node * SC, cnt * 16);
          prefetch_range(S.sB + (size_t)node * SC, cnt * 16);
        }
      }
    }
    // block-wide compaction of pushes, multipole items and direct items
    const bool push = (open | fdc) != 0 || ovp;
    const unsigned pb = __ballot_sync(FULL, push);
    const int nm = __popc(mac);
    int incl = nm;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += v;
    }
    const unsigned db = __ballot_sync(FULL, dir != 0 || ovd);
    if (lane == 31) {
      B.wcnt[warp][0] = __popc(pb);
      B.wcnt[warp][1] = incl;
      B.wcnt[warp][2] = __popc(db);
    }
    __syncthreads();
    int op = 0, oi = 0, od = 0, tp = 0, tm = 0, td = 0;
    for (int w = 0; w < NW; ++w) {
      const int c0 = B.wcnt[w][0], c1 = B.wcnt[w][1], c2 = B.wcnt[w][2];
      if (w < warp) {
        op += c0;
        oi += c1;
        od += c2;
      }
      tp += c0;
      tm += c1;
      td += c2;
    }
    if (top + tp > BHMC_BSTACK) {
      err = BHMC_ESTACK;
      break;
    }
    if (push)
      B.stk[top + op + __popc(pb & lt)] =
          make_uint2((unsigned)fc, open | (fdc << 4) | (onp << 8) | ((unsigned)(d + 1) << 12) |
                                       (ovp ? (1u << 17) : 0u));
    {
      int pos = oi + incl - nm;
      unsigned m = mac;
      while (m) {
        const int s = __ffs(m) - 1;
        m &= m - 1;
        B.mi[pos++] = ((unsigned)node << 4) | (emask << 2) | (unsigned)s;
      }
    }
    if (dir || ovd)
      B.di[od + __popc(db & lt)] = make_uint2((unsigned)node, ((unsigned)cnt << 4) | dir | (ovd ? (1u << 30) : 0u));
    accepted += nm;
    top += tp;
    __syncthreads();
    // next round: pop and prefetch its headers
    const int npop_n = min(top, G);
    uint2 e_n = make_uint2(0u, 0u);
    int4 b_n = make_int4(-1, 0, 0, 0);
    float4 a_n = make_float4(0.f, 0.f, 0.f, 0.f);
    if (g < npop_n) {
      e_n = B.stk[top - 1 - g];
      const int nn = (int)e_n.x + (tid & 7);
      b_n = ld_int4(S.nB + nn);
      a_n = ld_float4(S.nA + nn);
    }
    top -= npop_n;
    run_items(tm, td);
    // No barrier here: the next round writes the stack, the item lists and the
    // per-warp counts only after its first barrier, which every thread reaches
    // after finishing this round's items.
    e = e_n;
    b = b_n;
    a = a_n;
    npop = npop_n;
  }
  __syncthreads();
  // block reductions (result valid in thread 0).  The FP32 traversal's
  // compensated sums are added as float pairs, in FP32 arithmetic, which on
  // this part issues far faster than FP64; the FP64 traversal's and the
  // gradient sums are added in FP64.
  constexpr bool PAIRS = sizeof(Real) == 4 && !GRAD;
  if constexpr (PAIRS) {
    float h, l;
    acc.pair(h, l);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) df_add(h, l, __shfl_xor_sync(FULL, h, o), __shfl_xor_sync(FULL, l, o));
    if (lane == 0) {
      B.wsf[warp][0] = h;
      B.wsf[warp][1] = l;
    }
  } else {
    double v = acc.value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    double gg[8];
    if (GRAD) {
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        gg[4 * r] = ga.phi[r].value();
#pragma unroll
        for (int c = 0; c < 3; ++c) gg[4 * r + 1 + c] = (double)ga.g[r][c];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int u = 0; u < 8; ++u) gg[u] += __shfl_xor_sync(FULL, gg[u], o);
    }
    if (lane == 0) {
      B.wsum[warp] = v;
      if (GRAD) {
#pragma unroll
        for (int u = 0; u < 8; ++u) B.wg[warp][u] = gg[u];
      }
    }
  }
  const int r0 = __reduce_add_sync(FULL, visited), r1 = __reduce_add_sync(FULL, accepted);
  const int r2 = __reduce_add_sync(FULL, pairs), r3 = __reduce_add_sync(FULL, fp64);
  const int r4 = __reduce_max_sync(FULL, err);
  const int r5 = __any_sync(FULL, ovl) ? 1 : 0;
  if (lane == 0) {
    B.wred[warp][0] = r0;
    B.wred[warp][1] = r1;
    B.wred[warp][2] = r2;
    B.wred[warp][3] = r3;
    B.wred[warp][4] = r4;
    B.wred[warp][5] = r5;
  }
  __syncthreads();
  // warp 0 adds the per-warp results, one warp per lane
  if (warp == 0) {
    const bool in = lane < NW;
    const int c0 = __reduce_add_sync(FULL, in ? B.wred[lane][0] : 0);
    const int c1 = __reduce_add_sync(FULL, in ? B.wred[lane][1] : 0);
    const int c2 = __reduce_add_sync(FULL, in ? B.wred[lane][2] : 0);
    const int c3 = __reduce_add_sync(FULL, in ? B.wred[lane][3] : 0);
    const int c4 = __reduce_max_sync(FULL, in ? B.wred[lane][4] : 0);
    const unsigned c5 = __reduce_or_sync(FULL, in ? (unsigned)B.wred[lane][5] : 0u);
    double sum = 0.0;
    if constexpr (PAIRS) {
      float h = in ? B.wsf[lane][0] : 0.f, l = in ? B.wsf[lane][1] : 0.f;
#pragma unroll
      for (int o = BHMC_MAX_WARPS / 2; o > 0; o >>= 1)
        df_add(h, l, __shfl_xor_sync(FULL, h, o), __shfl_xor_sync(FULL, l, o));
      if (lane == 0) sum = (double)h + (double)l;
    }
    if (lane == 0) {
      out.sum = sum;
      for (int r = 0; r < 2; ++r) {
        out.phi[r] = 0.0;
        out.grad[r][0] = out.grad[r][1] = out.grad[r][2] = 0.0;
      }
      if (!PAIRS)
        for (int w = 0; w < NW; ++w) {
          out.sum += B.wsum[w];
          if (GRAD)
            for (int r = 0; r < 2; ++r) {
              out.phi[r] += B.wg[w][4 * r];
              for (int c = 0; c < 3; ++c) out.grad[r][c] += B.wg[w][4 * r + 1 + c];
            }
        }
      out.visited = c0;
      out.accepted = c1;
      out.pairs = c2;
      out.fp64 = c3;
      out.err = c4;
      out.overlap = (int)c5;
    }
  }
}

}  // namespace bhmc
