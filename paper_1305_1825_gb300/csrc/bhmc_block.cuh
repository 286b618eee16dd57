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

namespace bhmc {

struct BlockStore {
  uint2 stk[BHMC_BSTACK];
  unsigned mi[4 * 32 * BHMC_MAX_WARPS];  // node << 4 | excluded mask << 2 | point
  uint2 di[32 * BHMC_MAX_WARPS];         // {leaf, count << 4 | point mask}
  int wcnt[BHMC_MAX_WARPS][3];
  double wsum[BHMC_MAX_WARPS];
  int wred[BHMC_MAX_WARPS][5];
};

template <int P, typename Real, int LAYOUT>
__device__ void block_traverse(const SysDev& S, const TravPts& T, BlockStore& B, unsigned pmask,
                               int (*path)[BHMC_MAX_D + 1], TravOut& out) {
  const unsigned FULL = 0xffffffffu;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nth = blockDim.x, NW = nth >> 5, G = nth >> 3;
  const int g = tid >> 3;
  const unsigned lt = lanemask_lt();
  Acc<Real> acc;
  int visited = 0, accepted = 0, pairs = 0, fp64 = 0, err = 0;
  int cp = 1;
  while (cp < S.C) cp <<= 1;
  const int lg = 31 - __clz(cp);
  const int SC = S.C + 2;
  int top = 0, npop = 1;
  uint2 e = make_uint2(0u, g == 0 ? pmask : 0u);
  int4 b = make_int4(-1, 0, 0, 0);
  float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
  if (g == 0) {
    b = S.nB[tid & 7];
    a = S.nA[tid & 7];
  }
  int rounds = 0;
  while (npop > 0) {
    if (++rounds > (1 << 22)) {
      err = BHMC_ETIMEOUT;
      break;
    }
    const int node = (int)e.x + (tid & 7);
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
    // block-wide compaction of pushes, multipole items and direct items
    const bool push = (open | fdc) != 0;
    const unsigned pb = __ballot_sync(FULL, push);
    const int nm = __popc(mac);
    int incl = nm;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += v;
    }
    const unsigned db = __ballot_sync(FULL, dir != 0);
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
    if (push) B.stk[top + op + __popc(pb & lt)] = make_uint2((unsigned)fc, open | (fdc << 4));
    {
      int pos = oi + incl - nm;
      unsigned m = mac;
      while (m) {
        const int s = __ffs(m) - 1;
        m &= m - 1;
        B.mi[pos++] = ((unsigned)node << 4) | (emask << 2) | (unsigned)s;
      }
    }
    if (dir) B.di[od + __popc(db & lt)] = make_uint2((unsigned)node, ((unsigned)cnt << 4) | dir);
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
      b_n = S.nB[nn];
      a_n = S.nA[nn];
    }
    top -= npop_n;
    // first direct pass: issue its loads before the multipole work
    const int per = nth >> lg;
    const int kk = tid & (cp - 1);
    uint2 di0 = make_uint2(0u, 0u);
    float4 sa0 = make_float4(0.f, 0.f, 0.f, 0.f), sb0 = sa0;
    bool have0 = false;
    if ((tid >> lg) < td) {
      di0 = B.di[tid >> lg];
      if (kk < (int)(di0.y >> 4)) {
        const int slot = (int)di0.x * SC + kk;
        sa0 = S.sA[slot];
        sb0 = S.sB[slot];
        have0 = true;
      }
    }
    for (int k = tid; k < tm; k += nth) {
      const unsigned it = B.mi[k];
      const int s = (int)(it & 3u);
      const Real v = eval_item<P, Real, LAYOUT>(S, T, (int)(it >> 4), s, (it >> 2) & 3u);
      acc.add(sizeof(Real) == 4 ? (Real)(T.w[s] * (float)v) : (Real)(T.w64[s] * (double)v));
    }
    if (have0) direct_slot<Real>(S, T, sa0, sb0, di0.y & 15u, acc, pairs);
    for (int base = per; base < td; base += per) {
      const int item = base + (tid >> lg);
      if (item < td) {
        const uint2 di = B.di[item];
        if (kk < (int)(di.y >> 4)) {
          const int slot = (int)di.x * SC + kk;
          direct_slot<Real>(S, T, S.sA[slot], S.sB[slot], di.y & 15u, acc, pairs);
        }
      }
    }
    __syncthreads();
    e = e_n;
    b = b_n;
    a = a_n;
    npop = npop_n;
  }
  // block reductions (result valid in thread 0)
  double v = acc.value();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  const int r0 = __reduce_add_sync(FULL, visited), r1 = __reduce_add_sync(FULL, accepted);
  const int r2 = __reduce_add_sync(FULL, pairs), r3 = __reduce_add_sync(FULL, fp64);
  const int r4 = __reduce_max_sync(FULL, err);
  if (lane == 0) {
    B.wsum[warp] = v;
    B.wred[warp][0] = r0;
    B.wred[warp][1] = r1;
    B.wred[warp][2] = r2;
    B.wred[warp][3] = r3;
    B.wred[warp][4] = r4;
  }
  __syncthreads();
  if (tid == 0) {
    out.sum = 0.0;
    out.visited = out.accepted = out.pairs = out.fp64 = out.err = 0;
    for (int w = 0; w < NW; ++w) {
      out.sum += B.wsum[w];
      out.visited += B.wred[w][0];
      out.accepted += B.wred[w][1];
      out.pairs += B.wred[w][2];
      out.fp64 += B.wred[w][3];
      out.err = max(out.err, B.wred[w][4]);
    }
  }
}

}  // namespace bhmc
