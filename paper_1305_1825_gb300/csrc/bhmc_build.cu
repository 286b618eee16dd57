// bhmc_build.cu -- octree construction (Sec. 3.2), the stand-alone local
// adjustment kernel behind bhmc_commit_move (Sec. 3.3), and direct sums.
#include <algorithm>

#include "bhmc_build.cuh"
#include "bhmc_move.cuh"
#include "bhmc_forces.cuh"

namespace bhmc {

// Charges from the caller's AoS arrays into the SoA store; images of the
// mobile ions (position R^2 r/|r|^2, charge alpha q R/|r|) appended.
__global__ void k_init_charges(SysDev S, const double* q, const double* xyz, int* flags) {
  const int n_in = S.n_mob + S.n_fix;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_in; j += gridDim.x * blockDim.x) {
    const double r[3] = {xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2]};
    S.px[j] = r[0];
    S.py[j] = r[1];
    S.pz[j] = r[2];
    S.pq[j] = q[j];
    if (j < S.n_mob) {
      if (!shell_ok(S, r)) atomicMax(&flags[1], 1);
      if (S.images) {
        double im[3], qi;
        const int k = S.n_mob + S.n_fix + j;
        if (!image_of(S, r, q[j], im, &qi)) {
          atomicMax(&flags[0], 1);
          im[0] = im[1] = im[2] = 0.0;
          qi = 0.0;
        }
        S.px[k] = im[0];
        S.py[k] = im[1];
        S.pz[k] = im[2];
        S.pq[k] = qi;
      }
    }
  }
}

// Keys of every charge; perm lists the charges of the tree (with fixed_direct
// the fixed charges are left out and have no leaf).
__global__ void k_keys(SysDev S, int* perm, int* flags) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < S.n_tot; j += gridDim.x * blockDim.x) {
    const unsigned long long k = point_key(S, S.px[j], S.py[j], S.pz[j]);
    if (k == 0ULL) atomicMax(&flags[0], 1);
    S.ckey[j] = k;
    if (off_tree(S, j)) {
      S.leaf_of[j] = -1;
      S.slot_of[j] = -1;
    } else {
      perm[S.fixed_direct && j >= S.n_mob ? j - S.n_fix : j] = j;
    }
  }
}

__global__ void k_init_root(SysDev S, int* seg) {
  if (threadIdx.x < 8) {
    const int o = threadIdx.x;
    const float h = (float)(0.5 * S.root_side);
    const float c[3] = {(float)(S.root_lo[0] + 0.5 * S.root_side), (float)(S.root_lo[1] + 0.5 * S.root_side),
                        (float)(S.root_lo[2] + 0.5 * S.root_side)};
    S.nA[o] = o == 0 ? make_float4(c[0], c[1], c[2], h) : make_float4(0.f, 0.f, 0.f, 0.f);
    S.nB[o] = make_int4(-1, o == 0 ? S.n_tree : 0, o == 0 ? 1 : 0, 0);
    seg[o] = 0;
  }
  if (threadIdx.x == 0) {
    S.pool[0] = 1;
    S.pool[1] = 0;
    *S.energy = 0.0;
    *S.err = 0;
  }
}

// Split every cluster of `list` (one block each) into its eight octants: a
// stable partition of its segment of `perm` by the octant digit of the charge
// keys at depth+1; children get group base_group + blockIdx.x.
__global__ void __launch_bounds__(256) k_split_level(SysDev S, const int* list, int base_group, int depth,
                                                     int* perm, int* perm2, int* seg, int* next_flags) {
  __shared__ int counts[8], start[8], run[8], wtot[8][8];
  const int node = list[blockIdx.x];
  const int c0 = 8 * (base_group + blockIdx.x);
  const int st = seg[node];
  const int4 nb = S.nB[node];
  const int cnt = nb.y;
  const int sh = 3 * (S.Dmax - depth - 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < 8) counts[threadIdx.x] = 0;
  __syncthreads();
  for (int k = threadIdx.x; k < cnt; k += blockDim.x)
    atomicAdd(&counts[(int)((S.ckey[perm[st + k]] >> sh) & 7ULL)], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int o = 0; o < 8; ++o) {
      start[o] = s;
      run[o] = s;
      s += counts[o];
    }
  }
  __syncthreads();
  for (int base = 0; base < cnt; base += blockDim.x) {
    const int k = base + threadIdx.x;
    const bool valid = k < cnt;
    const int e = valid ? perm[st + k] : 0;
    const int o = valid ? (int)((S.ckey[e] >> sh) & 7ULL) : 8;
    int rank = 0;
    for (int d = 0; d < 8; ++d) {
      const unsigned m = __ballot_sync(0xffffffffu, o == d);
      if (o == d) rank = __popc(m & ((1u << lane) - 1u));
      if (lane == 0) wtot[warp][d] = __popc(m);
    }
    __syncthreads();
    if (valid) {
      int off = run[o];
      for (int w = 0; w < warp; ++w) off += wtot[w][o];
      perm2[st + off + rank] = e;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
      int add = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) add += wtot[w][threadIdx.x];
      run[threadIdx.x] += add;
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < cnt; k += blockDim.x) perm[st + k] = perm2[st + k];
  if (threadIdx.x < 8) {
    const int o = threadIdx.x;
    const float4 a = S.nA[node];
    const float hc = 0.5f * a.w;
    const unsigned long long key = ((unsigned long long)(unsigned)nb.w << 32) | (unsigned)nb.z;
    const unsigned long long ck = (key << 3) | (unsigned long long)o;
    S.nA[c0 + o] = make_float4((o & 1) ? a.x + hc : a.x - hc, (o & 2) ? a.y + hc : a.y - hc,
                               (o & 4) ? a.z + hc : a.z - hc, hc);
    S.nB[c0 + o] = make_int4(-1, counts[o], (int)(unsigned)(ck & 0xffffffffULL), (int)(unsigned)(ck >> 32));
    seg[c0 + o] = st + start[o];
    next_flags[8 * blockIdx.x + o] = (counts[o] > S.Cs && depth + 1 < S.Dmax) ? c0 + o : -1;
  }
  if (threadIdx.x == 0) S.nB[node].x = c0;
}

// Order-preserving compaction of the non-negative entries (one block).
__global__ void __launch_bounds__(1024) k_compact(const int* in, int n, int* out, int* n_out) {
  __shared__ int wsum[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = 0; base < n; base += blockDim.x) {
    const int k = base + threadIdx.x;
    const int v = k < n ? in[k] : -1;
    const unsigned m = __ballot_sync(0xffffffffu, v >= 0);
    if (lane == 0) wsum[warp] = __popc(m);
    __syncthreads();
    int off = carry;
    for (int w = 0; w < warp; ++w) off += wsum[w];
    if (v >= 0) out[off + __popc(m & ((1u << lane) - 1u))] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
      carry += t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_out = carry;
}

// Leaves receive their slots (charge positions as float pairs, charge, index).
__global__ void k_fill_leaves(SysDev S, int n_nodes, const int* perm, const int* seg, int* flags) {
  const int SC = S.C + 2;
  for (int nd = blockIdx.x * blockDim.x + threadIdx.x; nd < n_nodes; nd += gridDim.x * blockDim.x) {
    const int4 b = S.nB[nd];
    if (b.z == 0 && b.w == 0) continue;  // empty slot of the root group
    if (b.x >= 0) continue;
    if (b.y > S.C) {
      atomicMax(&flags[2], 1);
      continue;
    }
    for (int k = 0; k < b.y; ++k) {
      const int j = perm[seg[nd] + k];
      const float2 fx = split2(S.px[j]), fy = split2(S.py[j]), fz = split2(S.pz[j]);
      S.sA[nd * SC + k] = make_float4(fx.x, fy.x, fz.x, (float)S.pq[j]);
      S.sB[nd * SC + k] = make_float4(fx.y, fy.y, fz.y, __int_as_float(j));
      S.leaf_of[j] = nd;
      S.slot_of[j] = k;
    }
  }
}

// Leaf moments M_A^n = sum_{j in A} q_j (r_j - r_A)^n (Eq. 3.3) in FP64, one
// thread per (leaf, term), members in index order.
__global__ void k_moments_leaves(SysDev S, int n_nodes, const int* perm, const int* seg) {
  const long long total = (long long)n_nodes * S.K;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total;
       it += (long long)gridDim.x * blockDim.x) {
    const int nd = (int)(it / S.K), t = (int)(it - (long long)nd * S.K);
    const int4 b = S.nB[nd];
    if ((b.z == 0 && b.w == 0) || b.x >= 0) continue;
    const float4 c = S.nA[nd];
    int n1, n2, n3;
    term_exponents(t, n1, n2, n3);
    double M = 0.0;
    for (int k = 0; k < b.y; ++k) {
      const int j = perm[seg[nd] + k];
      M = __dadd_rn(M, mono_term(n1, n2, n3, S.pq[j], __dsub_rn(S.px[j], (double)c.x),
                                 __dsub_rn(S.py[j], (double)c.y), __dsub_rn(S.pz[j], (double)c.z)));
    }
    S.M64[(size_t)nd * S.K + t] = M;
    if (S.prec == BHMC_PREC_F32) S.M32[m32_index(S, nd, t)] = __double2float_rn(M);
  }
}

// Internal clusters of one level from their eight children (moments shifted
// from the child centre to the parent centre):
// M_P^n = sum_children sum_{m <= n} C(n, m) d^(n - m) M_child^m, d = r_child - r_P.
// Every component of d is +-h_c (the child's half side, a power of two), so each
// coefficient C(n1,m1) C(n2,m2) C(n3,m3) h_c^(|n| - |m|) with its sign is exact.
__global__ void k_moments_m2m(SysDev S, int node_begin, int node_end) {
  const long long total = (long long)(node_end - node_begin) * S.K;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total;
       it += (long long)gridDim.x * blockDim.x) {
    const int nd = node_begin + (int)(it / S.K), t = (int)(it % S.K);
    const int4 b = S.nB[nd];
    if ((b.z == 0 && b.w == 0) || b.x < 0) continue;
    int n1, n2, n3;
    term_exponents(t, n1, n2, n3);
    double hp[BHMC_MAX_P + 1];  // h_c^k
    hp[0] = 1.0;
    const double hc = (double)S.nA[b.x].w;
    for (int q = 1; q <= n1 + n2 + n3; ++q) hp[q] = hp[q - 1] * hc;
    double M = 0.0;
    for (int o = 0; o < 8; ++o) {
      const double* Mc = S.M64 + (size_t)(b.x + o) * S.K;
      for (int m1 = n1; m1 >= 0; --m1)
        for (int m2 = n2; m2 >= 0; --m2)
          for (int m3 = n3; m3 >= 0; --m3) {
            const int a1 = n1 - m1, a2 = n2 - m2, a3 = n3 - m3;
            // odd powers of a negative component flip the sign (child o lies
            // on the low side of axis k when bit k of o is clear)
            const bool neg = (((o & 1) == 0) && (a1 & 1)) != (((o & 2) == 0) && (a2 & 1)) !=
                             (((o & 4) == 0) && (a3 & 1));
            const double cf = (double)(binom(n1, m1) * binom(n2, m2) * binom(n3, m3)) * hp[a1 + a2 + a3];
            M = fma(neg ? -cf : cf, Mc[tidx(m1, m2, m3)], M);
          }
    }
    S.M64[(size_t)nd * S.K + t] = M;
    if (S.prec == BHMC_PREC_F32) S.M32[m32_index(S, nd, t)] = __double2float_rn(M);
  }
}

// Hard core of Eq. (2.1) in the initial configuration: flags[1] is set if two
// mobile ions are within the diameter.  One thread per mobile ion walks the
// clusters whose boxes come within the diameter of it (explicit stack of
// 8-sibling groups, bounded) and tests their leaves' mobile charges in FP64.
__global__ void k_hard_core_check(SysDev S, int* flags) {
  constexpr int kStack = 8 * (BHMC_MAX_D + 2);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < S.n_mob; j += gridDim.x * blockDim.x) {
    const double x[3] = {S.px[j], S.py[j], S.pz[j]};
    int stack[kStack];
    int top = 0;
    const int4 root = S.nB[0];
    bool hit = false;
    if (root.x < 0) {  // the root is a leaf
      for (int k = 0; k < root.y && !hit; ++k) {
        const int m = __float_as_int(S.sB[k].w);
        if (m >= S.n_mob || m == j) continue;
        const double dx = x[0] - S.px[m], dy = x[1] - S.py[m], dz = x[2] - S.pz[m];
        hit = (dx * dx + dy * dy) + dz * dz <= S.hc2;
      }
    } else {
      stack[top++] = root.x;
    }
    for (int guard = 0; top > 0 && !hit && guard < (1 << 22); ++guard) {
      const int g = stack[--top];
      for (int o = 0; o < 8 && !hit; ++o) {
        const int nd = g + o;
        const int4 b = S.nB[nd];
        if ((b.z == 0 && b.w == 0) || b.y == 0) continue;
        const float4 c = S.nA[nd];
        double e2 = 0.0;  // squared distance from x to the box (FP64, exact enough for pruning)
        for (int k = 0; k < 3; ++k) {
          const double ck = k == 0 ? c.x : (k == 1 ? c.y : c.z);
          const double e = fmax(fabs(x[k] - ck) - (double)c.w, 0.0);
          e2 += e * e;
        }
        if (e2 > S.hc2 * (1.0 + 1e-9)) continue;
        if (b.x >= 0) {
          if (top < kStack) stack[top++] = b.x;
          else atomicOr(&flags[3], 1);  // stack bound (never reached for valid trees)
          continue;
        }
        for (int k = 0; k < b.y && !hit; ++k) {
          const int m = __float_as_int(S.sB[nd * (S.C + 2) + k].w);
          if (m >= S.n_mob || m == j) continue;
          const double dx = x[0] - S.px[m], dy = x[1] - S.py[m], dz = x[2] - S.pz[m];
          hit = (dx * dx + dy * dy) + dz * dz <= S.hc2;
        }
      }
    }
    if (hit) atomicOr(&flags[1], 1);
  }
}

// Evaluation coefficients of every cluster in use (FP32 traversal).
__global__ void k_wmirror(SysDev S, int n_nodes) {
  const long long total = (long long)n_nodes * S.K;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total;
       it += (long long)gridDim.x * blockDim.x) {
    const int nd = (int)(it / S.K), t = (int)(it - (long long)nd * S.K);
    const int4 b = S.nB[nd];
    if (b.z == 0 && b.w == 0) continue;
    w_store(S, nd, t);
  }
}

// Stand-alone local adjustment (bhmc_commit_move): paths by descent from the root.
__global__ void __launch_bounds__(256) k_commit(SysDev S, int i, double bx, double by, double bz, int* status) {
  __shared__ MoveStore st;
  MoveSh& sh = st.sh;
  init_tables(sh, S.K);
  if (threadIdx.x == 0) {
    sh.i = i;
    sh.b[0] = bx;
    sh.b[1] = by;
    sh.b[2] = bz;
  }
  clear_paths(sh);
  __syncthreads();
  setup_move(S, sh);
  __syncthreads();
  if (threadIdx.x == 0) {
    const int o = sh.outcome;
    *status = o < 0 ? 0 : (o == BHMC_REJECT_DOMAIN ? BHMC_EDOMAIN : BHMC_EOVERLAP);
  }
  if (sh.outcome >= 0) return;
  complete_paths(S, sh);
  __syncthreads();
  if (threadIdx.x == 0) {
    sh.go = !capacity_violation(S, sh);
    if (!sh.go) *status = BHMC_ECAPACITY;
  }
  __syncthreads();
  if (!sh.go) return;
  commit_move_block(S, st);
}

// Direct O(N^2) energy, FP64: partial[block] = sum over its rows i of
// q_i sum_{j != i} q_j / r_ij.
__global__ void __launch_bounds__(256) k_direct_energy(const double* px, const double* py, const double* pz,
                                                       const double* pq, int n, double* partial) {
  __shared__ double red[8];
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double xi = px[i], yi = py[i], zi = pz[i];
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      const double dx = px[j] - xi, dy = py[j] - yi, dz = pz[j] - zi;
      s += pq[j] / sqrt(dx * dx + dy * dy + dz * dz);
    }
    acc += pq[i] * s;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    partial[blockIdx.x] = s;
  }
}

__global__ void k_interleave(SysDev S, double* q, double* xyz) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < S.n_tot; j += gridDim.x * blockDim.x) {
    if (q) q[j] = S.pq[j];
    if (xyz) {
      xyz[3 * j] = S.px[j];
      xyz[3 * j + 1] = S.py[j];
      xyz[3 * j + 2] = S.pz[j];
    }
  }
}

// ---------------------------------------------------------------------------
// Host-side launchers.
static inline int grid_for(long long n, int block) {
  long long g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 152 * 32) g = 152 * 32;
  return (int)g;
}

cudaError_t build_init_charges(const SysDev& S, const double* q, const double* xyz, int* flags,
                               cudaStream_t st) {
  k_init_charges<<<grid_for(S.n_mob + S.n_fix, 256), 256, 0, st>>>(S, q, xyz, flags);
  return cudaGetLastError();
}
cudaError_t build_keys(const SysDev& S, int* perm, int* flags, cudaStream_t st) {
  k_keys<<<grid_for(S.n_tot, 256), 256, 0, st>>>(S, perm, flags);
  return cudaGetLastError();
}
cudaError_t build_root(const SysDev& S, int* seg, cudaStream_t st) {
  k_init_root<<<1, 32, 0, st>>>(S, seg);
  return cudaGetLastError();
}
cudaError_t build_split_level(const SysDev& S, const int* list, int n_list, int base_group, int depth,
                              int* perm, int* perm2, int* seg, int* next_flags, cudaStream_t st) {
  k_split_level<<<n_list, 256, 0, st>>>(S, list, base_group, depth, perm, perm2, seg, next_flags);
  return cudaGetLastError();
}
cudaError_t build_compact(const int* in, int n, int* out, int* n_out, cudaStream_t st) {
  k_compact<<<1, 1024, 0, st>>>(in, n, out, n_out);
  return cudaGetLastError();
}
cudaError_t build_leaves_moments(const SysDev& S, int n_nodes, const int* perm, const int* seg, int* flags,
                                 const int* level_begin, int n_levels, cudaStream_t st) {
  k_fill_leaves<<<grid_for(n_nodes, 256), 256, 0, st>>>(S, n_nodes, perm, seg, flags);
  k_moments_leaves<<<grid_for((long long)n_nodes * S.K, 256), 256, 0, st>>>(S, n_nodes, perm, seg);
  // internal clusters bottom-up: level d occupies nodes [level_begin[d], level_begin[d + 1])
  for (int d = n_levels - 2; d >= 0; --d) {
    const int b = level_begin[d], e = level_begin[d + 1];
    k_moments_m2m<<<grid_for((long long)(e - b) * S.K, 256), 256, 0, st>>>(S, b, e);
  }
  return cudaGetLastError();
}
cudaError_t launch_wmirror(const SysDev& S, cudaStream_t st) {
  k_wmirror<<<grid_for((long long)S.node_cap * S.K, 256), 256, 0, st>>>(S, S.node_cap);
  return cudaGetLastError();
}
cudaError_t launch_hard_core_check(const SysDev& S, int* flags, cudaStream_t st) {
  if (S.hc2 > 0.0 && S.n_mob > 0) k_hard_core_check<<<grid_for(S.n_mob, 128), 128, 0, st>>>(S, flags);
  return cudaGetLastError();
}
// Radial counts of the mobile ions (Sec. 4 RDF and ICDF): r = sqrt((x x + y y)
// + z z), bin = floor((r - lo) / width), counted when 0 <= bin < nbins and
// lo <= r < hi (FP64, this operation order).
__global__ void k_radial_counts(SysDev S, int nbins, double lo, double hi, double width,
                                unsigned long long* counts, double* charge) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < S.n_mob; j += gridDim.x * blockDim.x) {
    const double x = S.px[j], y = S.py[j], z = S.pz[j];
    const double r = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
    if (!(r >= lo && r < hi)) continue;
    const double t = floor(__ddiv_rn(__dsub_rn(r, lo), width));
    if (!(t >= 0.0 && t < (double)nbins)) continue;
    const int k = (int)t;
    atomicAdd(&counts[k], 1ULL);
    atomicAdd(&charge[k], S.pq[j]);
  }
}
cudaError_t launch_radial_counts(const SysDev& S, int nbins, double lo, double hi, double width,
                                 unsigned long long* counts, double* charge, cudaStream_t st) {
  if (S.n_mob > 0) k_radial_counts<<<grid_for(S.n_mob, 256), 256, 0, st>>>(S, nbins, lo, hi, width, counts, charge);
  return cudaGetLastError();
}
cudaError_t launch_commit(const SysDev& S, int i, const double* b, int* status, cudaStream_t st) {
  k_commit<<<1, 128, 0, st>>>(S, i, b[0], b[1], b[2], status);
  return cudaGetLastError();
}
cudaError_t launch_direct_energy(const SysDev& S, double* partial, int nblk, cudaStream_t st) {
  k_direct_energy<<<nblk, 256, 0, st>>>(S.px, S.py, S.pz, S.pq, S.n_tot, partial);
  return cudaGetLastError();
}
cudaError_t launch_forces_push(const SysDev& S, const double* phi, const double* tgrad, const double* lam,
                               const double* psi, const double* src, double* dEdr, double* dEdq,
                               cudaStream_t st) {
  k_forces_push<<<grid_for(S.n_tot, 128), 128, 0, st>>>(S, phi, tgrad, lam, psi, src, dEdr, dEdq);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fixed charges held outside the tree (fixed_direct).  The traversal kernels
// of the energy and force passes see only the tree; these kernels add every
// pair that involves a fixed charge, exactly and in FP64.

// Sum over the block of v (valid in thread 0); every thread calls it.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

// Potential at fixed charge f = n_mob + blockIdx.x: the exact sum over every
// other charge.  Block (f, c) sums chunk c and adds it to phi[f] (phi may be
// null) and, times q_f, to qphi[blockIdx.x] (both zeroed by the caller).
__global__ void __launch_bounds__(256) k_fixed_targets(SysDev S, double* phi, double* qphi) {
  const int f = S.n_mob + blockIdx.x;
  const double x[3] = {S.px[f], S.py[f], S.pz[f]};
  double acc = 0.0;
  for (int j = blockIdx.y * blockDim.x + threadIdx.x; j < S.n_tot; j += gridDim.y * blockDim.x) {
    if (j == f) continue;
    const double e0 = __dsub_rn(S.px[j], x[0]), e1 = __dsub_rn(S.py[j], x[1]), e2 = __dsub_rn(S.pz[j], x[2]);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(e0, e0), __dmul_rn(e1, e1)), __dmul_rn(e2, e2));
    acc += __ddiv_rn(S.pq[j], __dsqrt_rn(r2));
  }
  const double t = block_sum(acc);
  if (threadIdx.x == 0) {
    atomicAdd(&qphi[blockIdx.x], S.pq[f] * t);
    if (phi) atomicAdd(&phi[f], t);
  }
}

// The fixed charges' exact potential at every charge of the tree, added to
// phi[j] (may be null; it holds the traversal's value), and
// sum_j q_j phi_fixed(r_j) added to *qsum.
__global__ void __launch_bounds__(256) k_fixed_tree_targets(SysDev S, double* phi, double* qsum) {
  double acc = 0.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < S.n_tot; j += gridDim.x * blockDim.x) {
    if (off_tree(S, j)) continue;
    const double x[3] = {S.px[j], S.py[j], S.pz[j]};
    const double v = fixed_phi(S, x, nullptr);
    if (phi) phi[j] += v;
    acc += S.pq[j] * v;
  }
  const double t = block_sum(acc);
  if (threadIdx.x == 0) atomicAdd(qsum, t);
}

// Adjoint of the pairs of fixed charge f = n_mob + blockIdx.x with every
// other charge: block (f, c) takes chunk c; target side phi_f and
// q_f grad phi_f added to phi[f] and tgrad[f] (zeroed by the caller), source
// side q_f / r to psi[j] and -q_f q_j (r_j - r_f) / r^3 to src[j].
__global__ void __launch_bounds__(256) k_forces_fixed(SysDev S, double* phi, double* tgrad, double* psi,
                                                      double* src) {
  const int f = S.n_mob + blockIdx.x;
  const double x[3] = {S.px[f], S.py[f], S.pz[f]};
  const double qf = S.pq[f];
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (int j = blockIdx.y * blockDim.x + threadIdx.x; j < S.n_tot; j += gridDim.y * blockDim.x) {
    if (j == f) continue;
    const double e[3] = {__dsub_rn(S.px[j], x[0]), __dsub_rn(S.py[j], x[1]), __dsub_rn(S.pz[j], x[2])};
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(e[0], e[0]), __dmul_rn(e[1], e[1])), __dmul_rn(e[2], e[2]));
    const double r = __dsqrt_rn(r2), r3 = __dmul_rn(r2, r);
    const double qj = S.pq[j];
    a[0] += __ddiv_rn(qj, r);
    atomicAdd(&psi[j], __ddiv_rn(qf, r));
    for (int c = 0; c < 3; ++c) {
      const double t = __ddiv_rn(e[c], r3);
      a[1 + c] += qj * t;
      atomicAdd(&src[3 * j + c], -qf * qj * t);
    }
  }
  for (int u = 0; u < 4; ++u) {
    const double t = block_sum(a[u]);
    if (threadIdx.x == 0) atomicAdd(u == 0 ? &phi[f] : &tgrad[3 * f + u - 1], u == 0 ? t : qf * t);
  }
}

// Adjoint of the pairs of every tree charge j with the fixed charges: target
// side phi_fixed(r_j) and q_j grad phi_fixed(r_j) added to phi[j] and
// tgrad[j] (which hold the traversal's values), source side q_j / r and
// -q_j q_f (r_f - r_j) / r^3 summed over each warp and added to psi[f], src[f].
__global__ void __launch_bounds__(256) k_forces_fixed_tree(SysDev S, double* phi, double* tgrad, double* psi,
                                                           double* src) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < S.n_tot; base += stride) {
    const int j = base + lane;
    const bool valid = j < S.n_tot && !off_tree(S, j);
    double x[3] = {0.0, 0.0, 0.0}, qj = 0.0;
    if (valid) {
      x[0] = S.px[j];
      x[1] = S.py[j];
      x[2] = S.pz[j];
      qj = S.pq[j];
      double g[3];
      phi[j] += fixed_phi(S, x, g);
      for (int c = 0; c < 3; ++c) tgrad[3 * j + c] += qj * g[c];
    }
    for (int f = S.n_mob; f < S.n_mob + S.n_fix; ++f) {
      double w[4] = {0.0, 0.0, 0.0, 0.0};
      if (valid) {
        const double e[3] = {__dsub_rn(S.px[f], x[0]), __dsub_rn(S.py[f], x[1]), __dsub_rn(S.pz[f], x[2])};
        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(e[0], e[0]), __dmul_rn(e[1], e[1])), __dmul_rn(e[2], e[2]));
        const double r = __dsqrt_rn(r2), r3 = __dmul_rn(r2, r);
        const double qq = __dmul_rn(qj, S.pq[f]);
        w[0] = __ddiv_rn(qj, r);
        for (int c = 0; c < 3; ++c) w[1 + c] = -__ddiv_rn(__dmul_rn(qq, e[c]), r3);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int u = 0; u < 4; ++u) w[u] += __shfl_xor_sync(FULL, w[u], o);
      if (lane == 0) {
        atomicAdd(&psi[f], w[0]);
        for (int c = 0; c < 3; ++c) atomicAdd(&src[3 * f + c], w[1 + c]);
      }
    }
  }
}

// Fixed charges held outside the tree: blocks per fixed charge so that the
// O(N) exact sums spread over the GPU.
static inline dim3 fixed_grid(const SysDev& S) {
  return dim3((unsigned)S.n_fix, (unsigned)std::max(1, std::min(64, (S.n_tot + 2047) / 2048)), 1);
}
static inline int tree_grid(const SysDev& S) { return std::max(1, std::min(152 * 8, (S.n_tot + 255) / 256)); }
cudaError_t launch_fixed_targets(const SysDev& S, double* phi, double* qphi, cudaStream_t st) {
  if (S.fixed_direct && S.n_fix > 0) {
    k_fixed_targets<<<fixed_grid(S), 256, 0, st>>>(S, phi, qphi);
    k_fixed_tree_targets<<<tree_grid(S), 256, 0, st>>>(S, phi, qphi + S.n_fix);
  }
  return cudaGetLastError();
}
cudaError_t launch_forces_fixed(const SysDev& S, double* phi, double* tgrad, double* psi, double* src,
                                cudaStream_t st) {
  if (S.fixed_direct && S.n_fix > 0) {
    k_forces_fixed<<<fixed_grid(S), 256, 0, st>>>(S, phi, tgrad, psi, src);
    k_forces_fixed_tree<<<tree_grid(S), 256, 0, st>>>(S, phi, tgrad, psi, src);
  }
  return cudaGetLastError();
}

cudaError_t launch_interleave(const SysDev& S, double* q, double* xyz, cudaStream_t st) {
  k_interleave<<<grid_for(S.n_tot, 256), 256, 0, st>>>(S, q, xyz);
  return cudaGetLastError();
}

}  // namespace bhmc
