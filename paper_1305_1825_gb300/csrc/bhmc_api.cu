// bhmc_api.cu -- host side of the C-ABI declared in include/bhmc.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "bhmc_build.cuh"
#include "bhmc_launch.cuh"

namespace bhmc {
struct DeltaOut {
  double dE;
  long long cnt[4];
  int status;
  int err;
};
struct MoveRec {
  long long i;
  double r[3];
  double dE;
  int outcome, flagged;
};
}  // namespace bhmc

using namespace bhmc;

static_assert(sizeof(MoveRec) == sizeof(bhmc_move_record), "record layout");

struct bhmc_ctx {
  bhmc_params P;
  SysDev S;
  cudaStream_t stream = nullptr;
  void* arena = nullptr;
  void* io = nullptr;       // device scratch for small results
  void* io_host = nullptr;  // pinned mirror
  int sticky = 0;
  bool borrowed = false;
  bool w_stale = true;  // W32 not refreshed since the moments last changed
  bhmc_counters last = {0, 0, 0, 0};  // counters of the last delta_energy / energy_counters
  void* rdf_buf = nullptr;            // radial sampling: running histogram and accumulators
};

struct bhmc_batch {
  std::vector<bhmc_ctx*> reps;
  SysDev* d_views = nullptr;
  BatchArgs* d_args = nullptr;
  BatchArgs* h_args = nullptr;
  unsigned long long* d_seeds = nullptr;
  int* d_order = nullptr;
  int* d_sched = nullptr;  // replica claim flags, cursor, head, per-SM slots (BatchArgs)
  int n_alone = -1;        // pairing of replicas per SM (BatchArgs::n_alone)
  bhmc_mc_stats* d_stats = nullptr;
  bhmc_mc_stats* h_stats = nullptr;
  int* d_errs = nullptr;  // each replica's error word after a batched launch
  int* h_errs = nullptr;
  cudaStream_t stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  int grid = 0;
  int warps = 1;
  int p = 4;
};

// Schedule words of a batched launch: claim flags, cursor, head, per-SM slots and heads.
static size_t sched_bytes(int n_rep) { return sizeof(int) * ((size_t)n_rep + 2 + 2 * BHMC_SM_IDS); }

#define CK(call)                              \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) return BHMC_ECUDA; \
  } while (0)

const char* bhmc_status_string(bhmc_status s) {
  switch (s) {
    case BHMC_OK: return "ok";
    case BHMC_EINVAL: return "invalid argument";
    case BHMC_EDOMAIN: return "position outside the root cube";
    case BHMC_EOVERLAP: return "position outside the confinement shell";
    case BHMC_ENOMEM: return "out of memory";
    case BHMC_ENOMEM_POOL: return "node pool exhausted";
    case BHMC_ECUDA: return "CUDA error";
    case BHMC_ETIMEOUT: return "bounded device loop exhausted";
    case BHMC_ESTATE: return "context holds an earlier device error";
    case BHMC_ECAPACITY: return "depth-Dmax cell over capacity";
    case BHMC_ESTACK: return "traversal stack overflow";
    case BHMC_ESCRATCH: return "problem larger than the call's fixed scratch";
    case BHMC_ENONFINITE: return "non-finite energy difference (FP32 expansion overflow)";
  }
  return "unknown status";
}

static bool pow2(double v) {
  int e;
  return v > 0.0 && std::frexp(v, &e) == 0.5;
}

static bhmc_status validate(const bhmc_params* P) {
  if (!P) return BHMC_EINVAL;
  if (!(P->lB > 0.0) || !(P->beta >= 0.0) || !(P->theta >= 0.0 && P->theta < 1.0)) return BHMC_EINVAL;
  if (P->p < 0 || P->p > BHMC_MAX_P) return BHMC_EINVAL;
  if (P->N0 < 0 || P->C < 2 || P->C > BHMC_MAX_C || P->Dmax < 1 || P->Dmax > BHMC_MAX_D) return BHMC_EINVAL;
  if (P->fixed_depth != 0 && P->fixed_depth != 1) return BHMC_EINVAL;
  if (!pow2(P->root_side)) return BHMC_EINVAL;
  const double hmin = std::ldexp(P->root_side, -P->Dmax);
  for (int a = 0; a < 3; ++a) {
    const double c = P->root_lo[a] / hmin;
    if (!std::isfinite(c) || c != std::floor(c)) return BHMC_EINVAL;
    // every cluster centre must be exact in FP32: |centre| / (hmin/2) < 2^24
    const double far = (std::fabs(P->root_lo[a]) + P->root_side) / (0.5 * hmin);
    if (far >= 16777216.0) return BHMC_EINVAL;
  }
  {
    int ex = 0;
    std::frexp(P->root_side, &ex);
    if (ex < -150 || ex > 150) return BHMC_EINVAL;  // keeps x * 2^Dmax / side exact for |x| >= 2^-823
  }
  if (P->shell && !(P->shell_rmin >= 0.0 && P->shell_rmax >= P->shell_rmin)) return BHMC_EINVAL;
  if (P->images && !(P->image_R > 0.0)) return BHMC_EINVAL;
  if (P->precision != BHMC_PREC_F32 && P->precision != BHMC_PREC_F64) return BHMC_EINVAL;
  if (P->layout != BHMC_LAYOUT_SOA && P->layout != BHMC_LAYOUT_AOS) return BHMC_EINVAL;
  if ((P->warps != 1 && P->warps != 2 && P->warps != 4 && P->warps != 8 && P->warps != 12 && P->warps != 16) ||
      P->warps > BHMC_MAX_WARPS)
    return BHMC_EINVAL;
  if (P->node_factor < 0.0) return BHMC_EINVAL;
  if (!(P->hard_core >= 0.0) || !std::isfinite(P->hard_core)) return BHMC_EINVAL;
  if (P->fixed_direct != 0 && P->fixed_direct != 1) return BHMC_EINVAL;
  if (P->round_limit < 0) return BHMC_EINVAL;
  return BHMC_OK;
}

// Map from moments to evaluation coefficients: multiplying the recurrence of
// Sec. 3.1 for T_n by r^(2k+1) gives polynomials N_n(R) = r^(2k+1) T_n(R),
//   N_0 = 1,  N_n = -[(2k - 1) sum_i R_i N_{n - e_i} + (k - 1) r^2 sum_i N_{n - 2 e_i}] / k,
// homogeneous of degree k; c(n, m) is the coefficient of R^m in N_n.
struct WMap {
  std::vector<int> row, col;
  std::vector<float> val;
};
static WMap wmap_make(int p) {
  const int K = nterms(p);
  std::vector<std::vector<double>> N(K, std::vector<double>(K, 0.0));
  std::vector<int> e1(K), e2(K), e3(K);
  for (int k = 0; k <= p; ++k)
    for (int n1 = k; n1 >= 0; --n1)
      for (int n2 = k - n1; n2 >= 0; --n2) {
        const int t = tidx(n1, n2, k - n1 - n2);
        e1[t] = n1;
        e2[t] = n2;
        e3[t] = k - n1 - n2;
      }
  N[0][0] = 1.0;
  for (int t = 1; t < K; ++t) {
    const int n[3] = {e1[t], e2[t], e3[t]};
    const int k = n[0] + n[1] + n[2];
    for (int i = 0; i < 3; ++i) {
      if (n[i] >= 1) {  // (2k - 1) R_i N_{n - e_i}
        int m[3] = {n[0], n[1], n[2]};
        m[i] -= 1;
        const int s = tidx(m[0], m[1], m[2]);
        for (int u = 0; u < K; ++u) {
          if (N[s][u] == 0.0) continue;
          int v[3] = {e1[u], e2[u], e3[u]};
          v[i] += 1;
          N[t][tidx(v[0], v[1], v[2])] -= (2.0 * k - 1.0) * N[s][u] / k;
        }
      }
      if (n[i] >= 2) {  // (k - 1) r^2 N_{n - 2 e_i}
        int m[3] = {n[0], n[1], n[2]};
        m[i] -= 2;
        const int s = tidx(m[0], m[1], m[2]);
        for (int u = 0; u < K; ++u) {
          if (N[s][u] == 0.0) continue;
          for (int j = 0; j < 3; ++j) {
            int v[3] = {e1[u], e2[u], e3[u]};
            v[j] += 2;
            N[t][tidx(v[0], v[1], v[2])] -= (k - 1.0) * N[s][u] / k;
          }
        }
      }
    }
  }
  WMap w;
  w.row.push_back(0);
  for (int m = 0; m < K; ++m) {
    for (int n = 0; n < K; ++n)
      if (N[n][m] != 0.0) {
        w.col.push_back(n);
        w.val.push_back((float)N[n][m]);
      }
    w.row.push_back((int)w.col.size());
  }
  return w;
}
static int wmap_nnz(int p) { return (int)wmap_make(p).col.size(); }

// Calls f(std::integral_constant<int, p>{}) for the multipole order p (0..10).
template <typename F>
static auto by_p(int p, F&& f) {
  switch (p) {
    case 0: return f(std::integral_constant<int, 0>{});
    case 1: return f(std::integral_constant<int, 1>{});
    case 2: return f(std::integral_constant<int, 2>{});
    case 3: return f(std::integral_constant<int, 3>{});
    case 4: return f(std::integral_constant<int, 4>{});
    case 5: return f(std::integral_constant<int, 5>{});
    case 6: return f(std::integral_constant<int, 6>{});
    case 7: return f(std::integral_constant<int, 7>{});
    case 8: return f(std::integral_constant<int, 8>{});
    case 9: return f(std::integral_constant<int, 9>{});
    default: return f(std::integral_constant<int, 10>{});
  }
}

template <typename T>
static T* carve(char*& cur, size_t n) {
  T* p = reinterpret_cast<T*>(cur);
  cur += (n * sizeof(T) + 255) & ~size_t(255);
  return p;
}

static size_t arena_bytes(const SysDev& S) {
  size_t b = 0;
  auto add = [&](size_t n) { b += (n + 255) & ~size_t(255); };
  add(4 * sizeof(double) * S.n_tot);  // px py pz pq
  add(sizeof(unsigned long long) * S.n_tot);
  add(2 * sizeof(int) * S.n_tot);
  add(sizeof(int) * S.n_tot);
  add(sizeof(float4) * S.node_cap);
  add(sizeof(int4) * S.node_cap);
  add(sizeof(float) * (size_t)S.node_cap * S.Kp);
  add(sizeof(float) * (size_t)S.node_cap * S.Kp);
  add(sizeof(double) * (size_t)S.node_cap * S.K);
  add(sizeof(int) * (S.K + 1));
  add(sizeof(int) * wmap_nnz(S.p));
  add(sizeof(float) * wmap_nnz(S.p));
  add(2 * sizeof(float4) * (size_t)S.node_cap * (S.C + 2));
  add(sizeof(int) * 2);
  add(sizeof(int) * S.group_cap);
  add(sizeof(double));
  add(sizeof(int));
  return b + 16 * 256;
}

static void carve_all(SysDev& S, char* base) {
  char* cur = base;
  S.px = carve<double>(cur, S.n_tot);
  S.py = carve<double>(cur, S.n_tot);
  S.pz = carve<double>(cur, S.n_tot);
  S.pq = carve<double>(cur, S.n_tot);
  S.ckey = carve<unsigned long long>(cur, S.n_tot);
  S.leaf_of = carve<int>(cur, S.n_tot);
  S.slot_of = carve<int>(cur, S.n_tot);
  S.order = carve<int>(cur, S.n_tot);
  S.nA = carve<float4>(cur, S.node_cap);
  S.nB = carve<int4>(cur, S.node_cap);
  S.M32 = carve<float>(cur, (size_t)S.node_cap * S.Kp);
  S.W32 = carve<float>(cur, (size_t)S.node_cap * S.Kp);
  S.M64 = carve<double>(cur, (size_t)S.node_cap * S.K);
  S.wrow = carve<int>(cur, S.K + 1);
  S.wcol = carve<int>(cur, wmap_nnz(S.p));
  S.wval = carve<float>(cur, wmap_nnz(S.p));
  S.sA = carve<float4>(cur, (size_t)S.node_cap * (S.C + 2));
  S.sB = carve<float4>(cur, (size_t)S.node_cap * (S.C + 2));
  S.pool = carve<int>(cur, 2);
  S.free_list = carve<int>(cur, S.group_cap);
  S.energy = carve<double>(cur, 1);
  S.err = carve<int>(cur, 1);
}

static void fill_view(SysDev& S, const bhmc_params* P, int64_t n_mob, int64_t n_fix) {
  std::memset(&S, 0, sizeof(S));
  S.n_mob = (int)n_mob;
  S.n_fix = (int)n_fix;
  S.n_tot = (int)(n_mob + n_fix + (P->images ? n_mob : 0));
  S.fixed_direct = P->fixed_direct ? 1 : 0;
  S.n_tree = S.n_tot - (S.fixed_direct ? (int)n_fix : 0);
  S.move_rounds = P->round_limit > 0 ? P->round_limit : (1 << 22);
  S.pass_pops = P->round_limit > 0 ? P->round_limit : (1 << 24);
  S.p = P->p;
  S.K = nterms(P->p);
  S.Kp = pad4(S.K);
  S.N0 = P->N0;
  S.C = P->C;
  S.Cs = P->fixed_depth ? 0 : P->C;
  S.Dmax = P->Dmax;
  S.images = P->images ? 1 : 0;
  S.shell = P->shell ? 1 : 0;
  S.prec = P->precision;
  S.layout = P->layout;
  S.lB = P->lB;
  S.beta = P->beta;
  S.theta2 = P->theta * P->theta;
  S.theta2f = (float)S.theta2;
  S.lBf = (float)P->lB;
  S.root_side = P->root_side;
  S.inv_hmin = std::ldexp(1.0, P->Dmax) / P->root_side;
  S.hmin_shift = std::ilogb(S.inv_hmin);
  for (int a = 0; a < 3; ++a) {
    S.root_lo[a] = P->root_lo[a];
    S.root_cell[a] = (long long)(P->root_lo[a] * S.inv_hmin);
  }
  S.rmin = P->shell_rmin;
  S.rmax = P->shell_rmax;
  S.img_R = P->image_R;
  S.rmin2 = S.rmin * S.rmin;
  S.rmax2 = S.rmax * S.rmax;
  S.img_R2 = S.img_R * S.img_R;
  S.hc2 = P->hard_core * P->hard_core;
  S.hc2f = (float)S.hc2;
  S.img_alpha = P->image_alpha;
  double f = 1.0 + std::max(1.0, 8.0 / P->C);
  if (P->fixed_depth) {  // a chain of clusters down to Dmax above every charge
    const int l8 = (int)std::floor(std::log((double)std::max<long long>(S.n_tot, 1)) / std::log(8.0));
    f = 8.0 * (double)std::max(1, P->Dmax - l8 + 1);
  }
  if (P->node_factor > 0.0) f = P->node_factor;
  long long cap = 64 + (long long)std::ceil(f * (double)S.n_tot);
  cap = (cap + 7) & ~7LL;
  S.node_cap = (int)std::min<long long>(cap, (1LL << 28));
  S.group_cap = S.node_cap / 8;
}

static bhmc_status ctx_check(bhmc_ctx* c) {
  if (!c) return BHMC_EINVAL;
  if (c->sticky) return BHMC_ESTATE;
  return BHMC_OK;
}

// Read the device error word; latch it.
static bhmc_status sync_err(bhmc_ctx* c) {
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
    c->sticky = BHMC_ECUDA;
    return BHMC_ECUDA;
  }
  int e = 0;
  if (cudaMemcpy(&e, c->S.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    c->sticky = BHMC_ECUDA;
    return BHMC_ECUDA;
  }
  if (e) {
    c->sticky = e;
    return (bhmc_status)e;
  }
  return BHMC_OK;
}

static bhmc_status build_tree(bhmc_ctx* c, const double* q, const double* xyz, int32_t flags) {
  SysDev& S = c->S;
  cudaStream_t st = c->stream;
  const int n_in = S.n_mob + S.n_fix;
  double *dq = nullptr, *dx = nullptr;
  int *perm = nullptr, *perm2 = nullptr, *seg = nullptr, *la = nullptr, *lb = nullptr, *fl = nullptr,
      *dflags = nullptr;
  bhmc_status rc = BHMC_OK;
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    if (!(flags & BHMC_DEVICE_PTRS)) {
      cudaFree(dq);
      cudaFree(dx);
    }
    cudaFree(perm);
    cudaFree(perm2);
    cudaFree(seg);
    cudaFree(la);
    cudaFree(lb);
    cudaFree(fl);
    cudaFree(dflags);
  };
  if (flags & BHMC_DEVICE_PTRS) {
    dq = const_cast<double*>(q);
    dx = const_cast<double*>(xyz);
  } else {
    if (cudaMalloc(&dq, sizeof(double) * n_in) != cudaSuccess ||
        cudaMalloc(&dx, sizeof(double) * 3 * n_in) != cudaSuccess) {
      cleanup();
      return BHMC_ENOMEM;
    }
    if (cudaMemcpyAsync(dq, q, sizeof(double) * n_in, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(dx, xyz, sizeof(double) * 3 * n_in, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      cleanup();
      return BHMC_ECUDA;
    }
  }
  if (cudaMalloc(&perm, sizeof(int) * S.n_tot) != cudaSuccess ||
      cudaMalloc(&perm2, sizeof(int) * S.n_tot) != cudaSuccess ||
      cudaMalloc(&seg, sizeof(int) * S.node_cap) != cudaSuccess ||
      cudaMalloc(&la, sizeof(int) * S.node_cap) != cudaSuccess ||
      cudaMalloc(&lb, sizeof(int) * S.node_cap) != cudaSuccess ||
      cudaMalloc(&fl, sizeof(int) * S.node_cap) != cudaSuccess ||
      cudaMalloc(&dflags, sizeof(int) * 8) != cudaSuccess) {
    cleanup();
    return BHMC_ENOMEM;
  }
  int hflags[8] = {0};
  bool ok = cudaMemsetAsync(dflags, 0, sizeof(int) * 8, st) == cudaSuccess &&
            build_init_charges(S, dq, dx, dflags, st) == cudaSuccess &&
            build_keys(S, perm, dflags, st) == cudaSuccess && build_root(S, seg, st) == cudaSuccess &&
            cudaMemcpyAsync(hflags, dflags, sizeof(int) * 8, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
            cudaStreamSynchronize(st) == cudaSuccess;
  if (!ok) {
    cleanup();
    return BHMC_ECUDA;
  }
  if (hflags[0]) rc = BHMC_EDOMAIN;
  else if (hflags[1]) rc = BHMC_EOVERLAP;
  if (rc != BHMC_OK) {
    cleanup();
    return rc;
  }
  int n_list = (S.n_tree > S.Cs && S.Dmax > 0) ? 1 : 0;
  int zero = 0;
  if (cudaMemcpyAsync(la, &zero, sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess) {
    cleanup();
    return BHMC_ECUDA;
  }
  int groups = 1;
  int* dcount = dflags + 4;
  // level d holds nodes [level_begin[d], level_begin[d + 1]); the root level is node 0
  std::vector<int> level_begin{0, 1};
  for (int depth = 0; n_list > 0; ++depth) {
    if (groups + n_list > S.group_cap) {
      cleanup();
      return BHMC_ENOMEM_POOL;
    }
    if (build_split_level(S, la, n_list, groups, depth, perm, perm2, seg, fl, st) != cudaSuccess ||
        build_compact(fl, 8 * n_list, lb, dcount, st) != cudaSuccess) {
      cleanup();
      return BHMC_ECUDA;
    }
    level_begin.back() = 8 * groups;
    groups += n_list;
    level_begin.push_back(8 * groups);
    if (cudaMemcpyAsync(&n_list, dcount, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      cleanup();
      return BHMC_ECUDA;
    }
    std::swap(la, lb);
  }
  if (cudaMemcpyAsync(S.pool, &groups, sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      (S.n_tree > 0 &&
       cudaMemcpyAsync(S.order, perm, sizeof(int) * S.n_tree, cudaMemcpyDeviceToDevice, st) != cudaSuccess) ||
      build_leaves_moments(S, 8 * groups, perm, seg, dflags, level_begin.data(), (int)level_begin.size(), st) != cudaSuccess ||
      launch_hard_core_check(S, dflags, st) != cudaSuccess ||
      cudaMemcpyAsync(hflags, dflags, sizeof(int) * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cleanup();
    return BHMC_ECUDA;
  }
  if (hflags[2]) rc = BHMC_ECAPACITY;
  else if (hflags[1]) rc = BHMC_EOVERLAP;  // hard-core overlap in the initial configuration
  cleanup();
  return rc;
}

// Small device/host scratch shared by the synchronous calls of one context.
struct IoBlock {
  DeltaOut delta;
  int status;
  int pad;
  bhmc_mc_stats stats;
  double energy;
};

static bhmc_status ctx_alloc(bhmc_ctx* c) {
  const size_t bytes = arena_bytes(c->S);
  if (cudaMalloc(&c->arena, bytes) != cudaSuccess) return BHMC_ENOMEM;
  carve_all(c->S, static_cast<char*>(c->arena));
  const WMap w = wmap_make(c->S.p);
  if (cudaMemcpyAsync(c->S.wrow, w.row.data(), sizeof(int) * w.row.size(), cudaMemcpyHostToDevice, c->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(c->S.wcol, w.col.data(), sizeof(int) * w.col.size(), cudaMemcpyHostToDevice, c->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(c->S.wval, w.val.data(), sizeof(float) * w.val.size(), cudaMemcpyHostToDevice,
                      c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return BHMC_ECUDA;
  if (cudaMalloc(&c->io, sizeof(IoBlock)) != cudaSuccess) return BHMC_ENOMEM;
  if (cudaMallocHost(&c->io_host, sizeof(IoBlock)) != cudaSuccess) return BHMC_ENOMEM;
  return BHMC_OK;
}

static void ctx_free(bhmc_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  cudaFree(c->arena);
  cudaFree(c->io);
  cudaFreeHost(c->io_host);
  cudaFree(c->rdf_buf);
  delete c;
}

// Radial sampling of a context (see bhmc_set_radial_sampling): buffers, the
// running histogram of the current configuration, zeroed accumulators.
static bhmc_status rdf_setup(bhmc_ctx* c, int32_t nbins, double r_lo, double r_hi, int64_t every) {
  bhmc_status rc = ctx_check(c);
  if (rc != BHMC_OK) return rc;
  if (nbins < 0 || nbins > (1 << 20) || every < 0) return BHMC_EINVAL;
  SysDev& S = c->S;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return BHMC_ECUDA;
  cudaFree(c->rdf_buf);
  c->rdf_buf = nullptr;
  S.rdf_nbins = 0;
  S.rdf_every = 0;
  S.rdf_run = S.rdf_acc = S.rdf_nsamp = nullptr;
  S.rdf_runq = S.rdf_accq = nullptr;
  if (nbins == 0) return BHMC_OK;
  if (!(r_hi > r_lo) || !std::isfinite(r_lo) || !std::isfinite(r_hi)) return BHMC_EINVAL;
  const size_t bytes = sizeof(unsigned long long) * (4 * (size_t)nbins + 1);
  if (cudaMalloc(&c->rdf_buf, bytes) != cudaSuccess) return BHMC_ENOMEM;
  char* b = static_cast<char*>(c->rdf_buf);
  const size_t nb = sizeof(unsigned long long) * (size_t)nbins;
  S.rdf_run = reinterpret_cast<unsigned long long*>(b);
  S.rdf_runq = reinterpret_cast<double*>(b + nb);
  S.rdf_acc = reinterpret_cast<unsigned long long*>(b + 2 * nb);
  S.rdf_accq = reinterpret_cast<double*>(b + 3 * nb);
  S.rdf_nsamp = reinterpret_cast<unsigned long long*>(b + 4 * nb);
  S.rdf_lo = r_lo;
  S.rdf_hi = r_hi;
  S.rdf_w = (r_hi - r_lo) / (double)nbins;
  if (cudaMemsetAsync(c->rdf_buf, 0, bytes, c->stream) != cudaSuccess ||
      launch_radial_counts(S, nbins, r_lo, r_hi, S.rdf_w, S.rdf_run, S.rdf_runq, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return BHMC_ECUDA;
  S.rdf_nbins = nbins;
  S.rdf_every = every;
  return BHMC_OK;
}

static bhmc_status rdf_read(bhmc_ctx* c, int64_t* counts, double* charge, int64_t* n_samples) {
  bhmc_status rc = ctx_check(c);
  if (rc != BHMC_OK) return rc;
  const SysDev& S = c->S;
  if (S.rdf_nbins <= 0) return BHMC_ESTATE;
  const int nb = S.rdf_nbins;
  std::vector<unsigned long long> hc(nb), hn(1);
  CK(cudaMemcpyAsync(hc.data(), S.rdf_acc, sizeof(unsigned long long) * nb, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(charge, S.rdf_accq, sizeof(double) * nb, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(hn.data(), S.rdf_nsamp, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < nb; ++k) counts[k] = (int64_t)hc[k];
  *n_samples = (int64_t)hn[0];
  return BHMC_OK;
}

static bhmc_status ctx_make(const bhmc_params* P, int64_t n_mob, int64_t n_fix, const double* q,
                            const double* xyz, int32_t flags, cudaStream_t stream, bhmc_ctx** out) {
  bhmc_status rc = validate(P);
  if (rc != BHMC_OK) return rc;
  if (n_mob < 0 || n_fix < 0 || n_mob + n_fix < 1 || !q || !xyz || !out) return BHMC_EINVAL;
  const long long n_tot = n_mob + n_fix + (P->images ? n_mob : 0);
  if (n_tot >= (1LL << 30)) return BHMC_EINVAL;
  bhmc_ctx* c = new (std::nothrow) bhmc_ctx();
  if (!c) return BHMC_ENOMEM;
  c->P = *P;
  c->stream = stream;
  fill_view(c->S, P, n_mob, n_fix);
  rc = ctx_alloc(c);
  if (rc == BHMC_OK) rc = build_tree(c, q, xyz, flags);
  if (rc != BHMC_OK) {
    ctx_free(c);
    return rc;
  }
  *out = c;
  return BHMC_OK;
}

extern "C" {

bhmc_status bhmc_create(const bhmc_params* params, int64_t n_mobile, int64_t n_fixed, const double* q,
                        const double* xyz, int32_t flags, void* cuda_stream, bhmc_ctx** out) {
  return ctx_make(params, n_mobile, n_fixed, q, xyz, flags, static_cast<cudaStream_t>(cuda_stream), out);
}

bhmc_status bhmc_destroy(bhmc_ctx* ctx) {
  if (!ctx) return BHMC_EINVAL;
  if (ctx->borrowed) return BHMC_EINVAL;
  ctx_free(ctx);
  return BHMC_OK;
}

bhmc_status bhmc_n_charges(const bhmc_ctx* ctx, int64_t* n) {
  if (!ctx || !n) return BHMC_EINVAL;
  *n = ctx->S.n_tot;
  return BHMC_OK;
}

bhmc_status bhmc_get_charges(bhmc_ctx* ctx, double* q, double* xyz, int32_t flags) {
  bhmc_status rc = ctx_check(ctx);
  if (rc != BHMC_OK) return rc;
  const SysDev& S = ctx->S;
  if (flags & BHMC_DEVICE_PTRS) {
    CK(launch_interleave(S, q, xyz, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return BHMC_OK;
  }
  std::vector<double> buf(4 * (size_t)S.n_tot);
  CK(cudaMemcpyAsync(buf.data(), S.px, sizeof(double) * S.n_tot, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(buf.data() + S.n_tot, S.py, sizeof(double) * S.n_tot, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(buf.data() + 2 * S.n_tot, S.pz, sizeof(double) * S.n_tot, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaMemcpyAsync(buf.data() + 3 * S.n_tot, S.pq, sizeof(double) * S.n_tot, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int j = 0; j < S.n_tot; ++j) {
    if (xyz) {
      xyz[3 * j] = buf[j];
      xyz[3 * j + 1] = buf[S.n_tot + j];
      xyz[3 * j + 2] = buf[2 * (size_t)S.n_tot + j];
    }
    if (q) q[j] = buf[3 * (size_t)S.n_tot + j];
  }
  return BHMC_OK;
}

static cudaError_t dispatch_delta(bhmc_ctx* c, int i, const double* b, DeltaOut* out) {
  return by_p(c->P.p, [&](auto PC) { return launch_delta<PC.value>(c->S, c->P.warps, i, b, out, c->stream); });
}

bhmc_status bhmc_delta_energy(bhmc_ctx* ctx, int64_t i, const double r_new[3], double* dE,
                              bhmc_counters* counters) {
  bhmc_status rc = ctx_check(ctx);
  if (rc != BHMC_OK) return rc;
  if (i < 0 || i >= ctx->S.n_mob || !r_new || !dE) return BHMC_EINVAL;
  IoBlock* dio = static_cast<IoBlock*>(ctx->io);
  IoBlock* hio = static_cast<IoBlock*>(ctx->io_host);
  CK(cudaMemsetAsync(&dio->delta, 0, sizeof(DeltaOut), ctx->stream));
  CK(dispatch_delta(ctx, (int)i, r_new, &dio->delta));
  CK(cudaMemcpyAsync(&hio->delta, &dio->delta, sizeof(DeltaOut), cudaMemcpyDeviceToHost, ctx->stream));
  rc = sync_err(ctx);
  if (rc != BHMC_OK) return rc;
  if (hio->delta.err) return (bhmc_status)hio->delta.err;
  if (hio->delta.status) return (bhmc_status)hio->delta.status;
  *dE = hio->delta.dE;
  ctx->last.visited = hio->delta.cnt[0];
  ctx->last.accepted = hio->delta.cnt[1];
  ctx->last.pairs = hio->delta.cnt[2];
  ctx->last.mac_fp64 = hio->delta.cnt[3];
  if (counters) *counters = ctx->last;
  return BHMC_OK;
}

bhmc_status bhmc_get_counters(bhmc_ctx* ctx, bhmc_counters* out) {
  if (!ctx || !out) return BHMC_EINVAL;
  *out = ctx->last;
  return BHMC_OK;
}

bhmc_status bhmc_get_positions(bhmc_ctx* ctx, double* xyz, int32_t flags) {
  if (!xyz) return BHMC_EINVAL;
  return bhmc_get_charges(ctx, nullptr, xyz, flags);
}

bhmc_status bhmc_commit_move(bhmc_ctx* ctx, int64_t i, const double r_new[3]) {
  bhmc_status rc = ctx_check(ctx);
  if (rc != BHMC_OK) return rc;
  ctx->w_stale = true;
  if (i < 0 || i >= ctx->S.n_mob || !r_new) return BHMC_EINVAL;
  IoBlock* dio = static_cast<IoBlock*>(ctx->io);
  IoBlock* hio = static_cast<IoBlock*>(ctx->io_host);
  CK(launch_commit(ctx->S, (int)i, r_new, &dio->status, ctx->stream));
  CK(cudaMemcpyAsync(&hio->status, &dio->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  rc = sync_err(ctx);
  if (rc != BHMC_OK) return rc;
  return (bhmc_status)hio->status;
}

static cudaError_t dispatch_step(bhmc_ctx* c, unsigned long long m, unsigned long long seed, double step,
                                 MoveRec* rec, bhmc_mc_stats* st) {
  return by_p(c->P.p, [&](auto PC) { return launch_step<PC.value>(c->S, c->P.warps, m, 0u, seed, step, rec, st, c->stream); });
}

bhmc_status bhmc_step_mc(bhmc_ctx* ctx, uint64_t n_moves, double step, uint64_t seed, uint64_t move0,
                         bhmc_mc_stats* stats, bhmc_move_record* records) {
  bhmc_status rc = ctx_check(ctx);
  if (rc != BHMC_OK) return rc;
  ctx->w_stale = true;
  if (!stats || !(step >= 0.0)) return BHMC_EINVAL;
  if (n_moves > 0 && ctx->S.n_mob < 1) return BHMC_EINVAL;  // no mobile ion to move
  IoBlock* dio = static_cast<IoBlock*>(ctx->io);
  IoBlock* hio = static_cast<IoBlock*>(ctx->io_host);
  MoveRec* drec = nullptr;
  if (records && n_moves) {
    if (cudaMalloc(&drec, sizeof(MoveRec) * n_moves) != cudaSuccess) return BHMC_ENOMEM;
  }
  CK(cudaMemsetAsync(&dio->stats, 0, sizeof(bhmc_mc_stats), ctx->stream));
  for (uint64_t t = 0; t < n_moves; ++t) {
    if (dispatch_step(ctx, move0 + t, seed, step, drec ? drec + t : nullptr, &dio->stats) != cudaSuccess) {
      cudaFree(drec);
      ctx->sticky = BHMC_ECUDA;
      return BHMC_ECUDA;
    }
  }
  CK(cudaMemcpyAsync(&hio->stats, &dio->stats, sizeof(bhmc_mc_stats), cudaMemcpyDeviceToHost, ctx->stream));
  if (drec)
    CK(cudaMemcpyAsync(records, drec, sizeof(MoveRec) * n_moves, cudaMemcpyDeviceToHost, ctx->stream));
  rc = sync_err(ctx);
  cudaFree(drec);
  if (rc != BHMC_OK) return rc;
  *stats = hio->stats;
  if (n_moves == 0) bhmc_get_energy(ctx, &stats->energy);
  return BHMC_OK;
}

bhmc_status bhmc_step_mc_spec(bhmc_ctx* ctx, uint64_t n_moves, double step, uint64_t seed, uint64_t move0,
                              int32_t proposals, bhmc_mc_stats* stats, bhmc_move_record* records) {
  bhmc_status rc = ctx_check(ctx);
  if (rc != BHMC_OK) return rc;
  ctx->w_stale = true;
  if (!stats || !(step >= 0.0) || proposals < 1 || proposals > BHMC_MAX_PROPOSALS) return BHMC_EINVAL;
  if (n_moves > 0 && ctx->S.n_mob < 1) return BHMC_EINVAL;
  IoBlock* dio = static_cast<IoBlock*>(ctx->io);
  IoBlock* hio = static_cast<IoBlock*>(ctx->io_host);
  MoveRec* drec = nullptr;
  if (records && n_moves) {
    if (cudaMalloc(&drec, sizeof(MoveRec) * n_moves) != cudaSuccess) return BHMC_ENOMEM;
  }
  CK(cudaMemsetAsync(&dio->stats, 0, sizeof(bhmc_mc_stats), ctx->stream));
  if (n_moves) {
    const cudaError_t e = by_p(ctx->P.p, [&](auto PC) {
      return launch_spec<PC.value>(ctx->S, ctx->P.warps, proposals, move0, n_moves, seed, step, drec,
                                   &dio->stats, ctx->stream);
    });
    if (e != cudaSuccess) {
      cudaFree(drec);
      ctx->sticky = BHMC_ECUDA;
      return BHMC_ECUDA;
    }
  }
  CK(cudaMemcpyAsync(&hio->stats, &dio->stats, sizeof(bhmc_mc_stats), cudaMemcpyDeviceToHost, ctx->stream));
  if (drec)
    CK(cudaMemcpyAsync(records, drec, sizeof(MoveRec) * n_moves, cudaMemcpyDeviceToHost, ctx->stream));
  rc = sync_err(ctx);
  cudaFree(drec);
  if (rc != BHMC_OK) return rc;
  *stats = hio->stats;
  if (n_moves == 0) bhmc_get_energy(ctx, &stats->energy);
  return BHMC_OK;
}

bhmc_status bhmc_step_mala(bhmc_ctx* ctx, uint64_t n_moves, double tau, uint64_t seed, uint64_t move0,
                           bhmc_mc_stats* stats, bhmc_move_record* records) {
  bhmc_status rc = ctx_check(ctx);
  if (rc != BHMC_OK) return rc;
  ctx->w_stale = true;
  if (!stats || !(tau > 0.0)) return BHMC_EINVAL;
  if (n_moves > 0 && ctx->S.n_mob < 1) return BHMC_EINVAL;
  IoBlock* dio = static_cast<IoBlock*>(ctx->io);
  IoBlock* hio = static_cast<IoBlock*>(ctx->io_host);
  MoveRec* drec = nullptr;
  if (records && n_moves) {
    if (cudaMalloc(&drec, sizeof(MoveRec) * n_moves) != cudaSuccess) return BHMC_ENOMEM;
  }
  CK(cudaMemsetAsync(&dio->stats, 0, sizeof(bhmc_mc_stats), ctx->stream));
  for (uint64_t t = 0; t < n_moves; ++t) {
    cudaError_t e;
    e = by_p(ctx->P.p, [&](auto PC) { return launch_step_mala<PC.value>(ctx->S, ctx->P.warps, move0 + t, 0u, seed, tau, drec ? drec + t : nullptr, &dio->stats, ctx->stream); });
    if (e != cudaSuccess) {
      cudaFree(drec);
      ctx->sticky = BHMC_ECUDA;
      return BHMC_ECUDA;
    }
  }
  CK(cudaMemcpyAsync(&hio->stats, &dio->stats, sizeof(bhmc_mc_stats), cudaMemcpyDeviceToHost, ctx->stream));
  if (drec)
    CK(cudaMemcpyAsync(records, drec, sizeof(MoveRec) * n_moves, cudaMemcpyDeviceToHost, ctx->stream));
  rc = sync_err(ctx);
  cudaFree(drec);
  if (rc != BHMC_OK) return rc;
  *stats = hio->stats;
  return BHMC_OK;
}

// Radial counts of one or more systems into host arrays (accumulated).
static bhmc_status radial_impl(bhmc_ctx* const* ctxs, int n, int32_t nbins, double r_lo, double r_hi,
                               int64_t* counts, double* charge) {
  if (!ctxs || n < 1 || nbins < 1 || nbins > (1 << 24) || !counts || !charge || !(r_hi > r_lo) ||
      !std::isfinite(r_lo) || !std::isfinite(r_hi))
    return BHMC_EINVAL;
  for (int k = 0; k < n; ++k) {
    bhmc_status rc = ctx_check(ctxs[k]);
    if (rc != BHMC_OK) return rc;
  }
  const double width = (r_hi - r_lo) / (double)nbins;
  cudaStream_t st = ctxs[0]->stream;
  unsigned long long* dc = nullptr;
  double* dq = nullptr;
  if (cudaMalloc(&dc, sizeof(unsigned long long) * nbins) != cudaSuccess) return BHMC_ENOMEM;
  if (cudaMalloc(&dq, sizeof(double) * nbins) != cudaSuccess) {
    cudaFree(dc);
    return BHMC_ENOMEM;
  }
  std::vector<unsigned long long> hc(nbins);
  std::vector<double> hq(nbins);
  bool ok = cudaMemsetAsync(dc, 0, sizeof(unsigned long long) * nbins, st) == cudaSuccess &&
            cudaMemsetAsync(dq, 0, sizeof(double) * nbins, st) == cudaSuccess;
  for (int k = 0; ok && k < n; ++k)
    ok = launch_radial_counts(ctxs[k]->S, nbins, r_lo, r_hi, width, dc, dq, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(hc.data(), dc, sizeof(unsigned long long) * nbins, cudaMemcpyDeviceToHost, st) ==
                 cudaSuccess &&
       cudaMemcpyAsync(hq.data(), dq, sizeof(double) * nbins, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
       cudaStreamSynchronize(st) == cudaSuccess;
  cudaFree(dc);
  cudaFree(dq);
  if (!ok) return BHMC_ECUDA;
  for (int k = 0; k < nbins; ++k) {
    counts[k] += (int64_t)hc[k];
    charge[k] += hq[k];
  }
  return BHMC_OK;
}

bhmc_status bhmc_radial_counts(bhmc_ctx* ctx, int32_t nbins, double r_lo, double r_hi, int64_t* counts,
                               double* charge) {
  return radial_impl(&ctx, 1, nbins, r_lo, r_hi, counts, charge);
}

bhmc_status bhmc_set_radial_sampling(bhmc_ctx* ctx, int32_t nbins, double r_lo, double r_hi, int64_t every) {
  if (ctx && ctx->borrowed) return BHMC_EINVAL;  // a replica: use bhmc_batch_set_radial_sampling
  return rdf_setup(ctx, nbins, r_lo, r_hi, every);
}

bhmc_status bhmc_get_radial_samples(bhmc_ctx* ctx, int64_t* counts, double* charge, int64_t* n_samples) {
  if (!counts || !charge || !n_samples) return BHMC_EINVAL;
  return rdf_read(ctx, counts, charge, n_samples);
}

bhmc_status bhmc_radial_profiles(int32_t nbins, double r_lo, double r_hi, const int64_t* counts,
                                 const double* charge, int64_t n_samples, double q_fixed, double* r_mid, double* g,
                                 double* r_out, double* Q) {
  if (nbins < 1 || !(r_hi > r_lo) || n_samples < 1 || !counts || !charge || !r_mid || !g || !r_out || !Q)
    return BHMC_EINVAL;
  const double w = (r_hi - r_lo) / (double)nbins;
  double total = 0.0, q = q_fixed;
  for (int k = 0; k < nbins; ++k) {
    const double a = r_lo + k * w, b = r_lo + (k + 1) * w;
    const double vol = 4.0 / 3.0 * 3.14159265358979323846 * (b * b * b - a * a * a);
    g[k] = ((double)counts[k] / (double)n_samples) / vol;  // mean number density of the bin
    total += g[k];
    q += charge[k] / (double)n_samples;
    r_mid[k] = 0.5 * (a + b);
    r_out[k] = b;
    Q[k] = q;
  }
  for (int k = 0; k < nbins; ++k) g[k] = total > 0.0 ? g[k] / total : 0.0;
  return BHMC_OK;
}

bhmc_status bhmc_get_energy(bhmc_ctx* ctx, double* E) {
  if (!ctx || !E) return BHMC_EINVAL;
  CK(cudaMemcpyAsync(E, ctx->S.energy, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return BHMC_OK;
}

bhmc_status bhmc_set_energy(bhmc_ctx* ctx, double E) {
  bhmc_status rc = ctx_check(ctx);
  if (rc != BHMC_OK) return rc;
  IoBlock* hio = static_cast<IoBlock*>(ctx->io_host);
  hio->energy = E;
  CK(cudaMemcpyAsync(ctx->S.energy, &hio->energy, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return BHMC_OK;
}

static cudaError_t dispatch_energy(bhmc_ctx* c, int grid, double* partial, double* phi, int* err,
                                   unsigned long long* cnt) {
  const int w = BHMC_ENERGY_WARPS;
  return by_p(c->P.p, [&](auto PC) { return launch_energy<PC.value>(c->S, w, grid, partial, phi, err, cnt, c->stream); });
}

static bhmc_status energy_impl(bhmc_ctx* ctx, double* E, double* phi_out, int32_t flags,
                               bhmc_counters* total = nullptr) {
  bhmc_status rc = ctx_check(ctx);
  if (rc != BHMC_OK) return rc;
  const int warps = BHMC_ENERGY_WARPS;  // each warp evaluates 32 targets at a time
  int grid = (ctx->S.n_tree + 32 * warps - 1) / (32 * warps);
  grid = std::max(1, std::min(grid, 152 * 16));
  // one partial per warp, then q_f phi_f of each fixed charge held outside the
  // tree and sum_j q_j phi_fixed(r_j) over the tree's charges
  const int n_off = ctx->S.fixed_direct && ctx->S.n_fix > 0 ? ctx->S.n_fix + 1 : 0;
  double* partial = nullptr;
  int* derr = nullptr;  // error flag, then three counters (8-byte aligned)
  if (cudaMalloc(&partial, sizeof(double) * ((size_t)grid * warps + n_off)) != cudaSuccess) return BHMC_ENOMEM;
  if (cudaMalloc(&derr, 32) != cudaSuccess) {
    cudaFree(partial);
    return BHMC_ENOMEM;
  }
  unsigned long long* dcnt = total ? reinterpret_cast<unsigned long long*>(derr) + 1 : nullptr;
  unsigned long long hcnt[3] = {0, 0, 0};
  double* dphi = nullptr;
  if (phi_out) {
    if (flags & BHMC_DEVICE_PTRS) {
      dphi = phi_out;
    } else if (cudaMalloc(&dphi, sizeof(double) * ctx->S.n_tot) != cudaSuccess) {
      cudaFree(partial);
      cudaFree(derr);
      return BHMC_ENOMEM;
    }
  }
  std::vector<double> h((size_t)grid * warps + n_off);
  int herr = 0;
  // the FP32 pass at p >= 6 evaluates from W32, refreshed here after moves
  const bool wform = ctx->S.prec == BHMC_PREC_F32 && ctx->S.p >= 6;
  double* qphi = partial + (size_t)grid * warps;
  bool ok = (!wform || !ctx->w_stale || launch_wmirror(ctx->S, ctx->stream) == cudaSuccess) &&
            cudaMemsetAsync(derr, 0, 32, ctx->stream) == cudaSuccess &&
            dispatch_energy(ctx, grid, partial, dphi, derr, dcnt) == cudaSuccess &&
            (n_off == 0 ||
             (cudaMemsetAsync(qphi, 0, sizeof(double) * n_off, ctx->stream) == cudaSuccess &&
              (!dphi || cudaMemsetAsync(dphi + ctx->S.n_mob, 0, sizeof(double) * ctx->S.n_fix, ctx->stream) == cudaSuccess) &&
              launch_fixed_targets(ctx->S, dphi, qphi, ctx->stream) == cudaSuccess)) &&
            cudaMemcpyAsync(h.data(), partial, sizeof(double) * h.size(), cudaMemcpyDeviceToHost,
                            ctx->stream) == cudaSuccess &&
            cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream) == cudaSuccess;
  if (ok && dcnt)
    ok = cudaMemcpyAsync(hcnt, dcnt, sizeof hcnt, cudaMemcpyDeviceToHost, ctx->stream) == cudaSuccess;
  if (ok && phi_out && !(flags & BHMC_DEVICE_PTRS))
    ok = cudaMemcpyAsync(phi_out, dphi, sizeof(double) * ctx->S.n_tot, cudaMemcpyDeviceToHost, ctx->stream) ==
         cudaSuccess;
  ok = ok && cudaStreamSynchronize(ctx->stream) == cudaSuccess;
  cudaFree(partial);
  cudaFree(derr);
  if (phi_out && !(flags & BHMC_DEVICE_PTRS)) cudaFree(dphi);
  if (!ok) return BHMC_ECUDA;
  if (herr) return (bhmc_status)herr;
  ctx->w_stale = false;
  double s = 0.0;
  for (double v : h) s += v;
  if (E) *E = 0.5 * ctx->S.lB * s;
  if (total) {
    total->visited = (int64_t)hcnt[0];
    total->accepted = (int64_t)hcnt[1];
    total->pairs = (int64_t)hcnt[2];
    total->mac_fp64 = 0;
    ctx->last = *total;
  }
  return BHMC_OK;
}

bhmc_status bhmc_energy_counters(bhmc_ctx* ctx, double* E, bhmc_counters* total) {
  if (!E || !total) return BHMC_EINVAL;
  return energy_impl(ctx, E, nullptr, 0, total);
}

bhmc_status bhmc_energy(bhmc_ctx* ctx, double* E) {
  if (!E) return BHMC_EINVAL;
  return energy_impl(ctx, E, nullptr, 0);
}

bhmc_status bhmc_potentials(bhmc_ctx* ctx, double* phi, int32_t flags) {
  if (!phi) return BHMC_EINVAL;
  return energy_impl(ctx, nullptr, phi, flags);
}

bhmc_status bhmc_forces(bhmc_ctx* ctx, double* dEdr, double* dEdq, int32_t flags) {
  bhmc_status rc = ctx_check(ctx);
  if (rc != BHMC_OK) return rc;
  if (!dEdr || !dEdq) return BHMC_EINVAL;
  const SysDev& S = ctx->S;
  const size_t n = (size_t)S.n_tot;
  const size_t nl = (size_t)S.node_cap * S.K;
  // scratch: phi, target gradients, cluster adjoints, direct source terms, outputs
  const size_t doubles = n + 3 * n + nl + n + 3 * n + (flags & BHMC_DEVICE_PTRS ? 0 : 4 * n);
  double* buf = nullptr;
  int* derr = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * doubles) != cudaSuccess) return BHMC_ENOMEM;
  if (cudaMalloc(&derr, sizeof(int)) != cudaSuccess) {
    cudaFree(buf);
    return BHMC_ENOMEM;
  }
  double* phi = buf;
  double* tg = phi + n;
  double* lam = tg + 3 * n;
  double* psi = lam + nl;
  double* src = psi + n;
  double* odr = (flags & BHMC_DEVICE_PTRS) ? dEdr : src + 3 * n;
  double* odq = (flags & BHMC_DEVICE_PTRS) ? dEdq : odr + 3 * n;
  const int grid = (int)std::max<size_t>(1, std::min<size_t>(((size_t)S.n_tree + 127) / 128, 152 * 16));
  cudaError_t e = cudaMemsetAsync(lam, 0, sizeof(double) * (nl + 4 * n), ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(int), ctx->stream);
  if (e == cudaSuccess && S.fixed_direct && S.n_fix > 0) {
    // the fixed charges outside the tree accumulate their target side
    e = cudaMemsetAsync(phi + S.n_mob, 0, sizeof(double) * S.n_fix, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(tg + 3 * (size_t)S.n_mob, 0, sizeof(double) * 3 * S.n_fix, ctx->stream);
  }
  if (e == cudaSuccess) {
    e = by_p(ctx->P.p, [&](auto PC) { return launch_forces<PC.value>(S, grid, phi, tg, lam, psi, src, derr, ctx->stream); });
  }
  if (e == cudaSuccess) e = launch_forces_fixed(S, phi, tg, psi, src, ctx->stream);
  if (e == cudaSuccess) e = launch_forces_push(S, phi, tg, lam, psi, src, odr, odq, ctx->stream);
  int herr = 0;
  if (e == cudaSuccess && !(flags & BHMC_DEVICE_PTRS)) {
    e = cudaMemcpyAsync(dEdr, odr, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dEdq, odq, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(buf);
  cudaFree(derr);
  if (e != cudaSuccess) return BHMC_ECUDA;
  return herr ? (bhmc_status)herr : BHMC_OK;
}

bhmc_status bhmc_energy_direct(bhmc_ctx* ctx, double* E) {
  bhmc_status rc = ctx_check(ctx);
  if (rc != BHMC_OK) return rc;
  if (!E) return BHMC_EINVAL;
  const int nblk = std::max(1, std::min((ctx->S.n_tot + 255) / 256, 152 * 8));
  double* partial = nullptr;
  if (cudaMalloc(&partial, sizeof(double) * nblk) != cudaSuccess) return BHMC_ENOMEM;
  std::vector<double> h(nblk);
  bool ok = launch_direct_energy(ctx->S, partial, nblk, ctx->stream) == cudaSuccess &&
            cudaMemcpyAsync(h.data(), partial, sizeof(double) * nblk, cudaMemcpyDeviceToHost, ctx->stream) ==
                cudaSuccess &&
            cudaStreamSynchronize(ctx->stream) == cudaSuccess;
  cudaFree(partial);
  if (!ok) return BHMC_ECUDA;
  double s = 0.0;
  for (double v : h) s += v;
  *E = 0.5 * ctx->S.lB * s;
  return BHMC_OK;
}

bhmc_status bhmc_export_tree(bhmc_ctx* ctx, int64_t* rows, int64_t max_rows, int64_t* members,
                             int64_t max_members, double* moments, int64_t* n_rows) {
  bhmc_status rc = ctx_check(ctx);
  if (rc != BHMC_OK) return rc;
  if (!rows || !members || !n_rows) return BHMC_EINVAL;
  const SysDev& S = ctx->S;
  int pool[2];
  CK(cudaMemcpyAsync(pool, S.pool, sizeof(pool), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const size_t nn = 8 * (size_t)pool[0];
  const int SC = S.C + 2;
  std::vector<int4> nb(nn);
  std::vector<float4> sb(nn * SC);
  std::vector<double> M;
  CK(cudaMemcpyAsync(nb.data(), S.nB, sizeof(int4) * nn, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(sb.data(), S.sB, sizeof(float4) * nn * SC, cudaMemcpyDeviceToHost, ctx->stream));
  if (moments) {
    M.resize(nn * S.K);
    CK(cudaMemcpyAsync(M.data(), S.M64, sizeof(double) * nn * S.K, cudaMemcpyDeviceToHost, ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  int64_t nr = 0, nm = 0;
  std::vector<int> stack{0};
  while (!stack.empty()) {
    const int a = stack.back();
    stack.pop_back();
    const int4 b = nb[a];
    const unsigned long long key = ((unsigned long long)(unsigned)b.w << 32) | (unsigned)b.z;
    if (nr >= max_rows) return BHMC_EINVAL;
    int depth = 0;
    for (unsigned long long k = key; k > 1; k >>= 3) ++depth;
    rows[4 * nr + 0] = depth;
    rows[4 * nr + 1] = (int64_t)key;
    rows[4 * nr + 2] = b.x < 0 ? 1 : 0;
    rows[4 * nr + 3] = b.y;
    if (moments)
      for (int t = 0; t < S.K; ++t) moments[nr * S.K + t] = M[(size_t)a * S.K + t];
    ++nr;
    if (b.x < 0) {
      if (nm + b.y > max_members) return BHMC_EINVAL;
      for (int k = 0; k < b.y; ++k) {
        const float w = sb[(size_t)a * SC + k].w;
        int j;
        std::memcpy(&j, &w, sizeof(int));
        members[nm + k] = j;
      }
      std::sort(members + nm, members + nm + b.y);
      nm += b.y;
    } else {
      for (int o = 7; o >= 0; --o) stack.push_back(b.x + o);
    }
  }
  *n_rows = nr;
  return BHMC_OK;
}

// ---------------------------------------------------------------------------
bhmc_status bhmc_batch_create(int32_t n_rep, const bhmc_params* params, const int64_t* n_mobile,
                              const int64_t* n_fixed, const double* const* q, const double* const* xyz,
                              int32_t flags, void* cuda_stream, bhmc_batch** out) {
  if (n_rep < 1 || !params || !n_mobile || !n_fixed || !q || !xyz || !out) return BHMC_EINVAL;
  bhmc_status rc = validate(params);
  if (rc != BHMC_OK) return rc;
  bhmc_batch* B = new (std::nothrow) bhmc_batch();
  if (!B) return BHMC_ENOMEM;
  B->stream = static_cast<cudaStream_t>(cuda_stream);
  B->warps = params->warps;
  B->p = params->p;
  for (int r = 0; r < n_rep; ++r) {
    bhmc_ctx* c = nullptr;
    rc = ctx_make(params, n_mobile[r], n_fixed[r], q[r], xyz[r], flags, B->stream, &c);
    if (rc != BHMC_OK) {
      bhmc_batch_destroy(B);
      return rc;
    }
    c->borrowed = true;
    B->reps.push_back(c);
  }
  std::vector<SysDev> views(n_rep);
  for (int r = 0; r < n_rep; ++r) views[r] = B->reps[r]->S;
  if (cudaMalloc(&B->d_views, sizeof(SysDev) * n_rep) != cudaSuccess ||
      cudaMalloc(&B->d_args, sizeof(BatchArgs)) != cudaSuccess ||
      cudaMallocHost(&B->h_args, sizeof(BatchArgs)) != cudaSuccess ||
      cudaMalloc(&B->d_seeds, sizeof(unsigned long long) * n_rep) != cudaSuccess ||
      cudaMalloc(&B->d_sched, sched_bytes(n_rep)) != cudaSuccess ||
      cudaMalloc(&B->d_order, sizeof(int) * n_rep) != cudaSuccess ||
      cudaMalloc(&B->d_stats, sizeof(bhmc_mc_stats) * n_rep) != cudaSuccess ||
      cudaMallocHost(&B->h_stats, sizeof(bhmc_mc_stats) * n_rep) != cudaSuccess ||
      cudaMalloc(&B->d_errs, sizeof(int) * n_rep) != cudaSuccess ||
      cudaMallocHost(&B->h_errs, sizeof(int) * n_rep) != cudaSuccess) {
    bhmc_batch_destroy(B);
    return BHMC_ENOMEM;
  }
  // Blocks take replicas largest first: the first block on each SM gets one of
  // the largest systems, the second blocks (on some SMs) the smallest, which
  // finish early and leave their SM to the large chain.
  std::vector<int> order(n_rep);
  for (int r = 0; r < n_rep; ++r) order[r] = r;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return views[x].n_tot > views[y].n_tot; });
  if (cudaMemcpy(B->d_order, order.data(), sizeof(int) * n_rep, cudaMemcpyHostToDevice) != cudaSuccess) {
    bhmc_batch_destroy(B);
    return BHMC_ECUDA;
  }
  if (cudaMemcpy(B->d_views, views.data(), sizeof(SysDev) * n_rep, cudaMemcpyHostToDevice) != cudaSuccess) {
    bhmc_batch_destroy(B);
    return BHMC_ECUDA;
  }
  int occ = 0;
  occ = by_p(B->p, [&](auto PC) { return batch_occupancy<PC.value>(views[0], B->warps); });
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  B->grid = std::max(1, std::min(n_rep, std::max(1, occ) * std::max(1, sms)));
  if (occ >= 2 && sms < n_rep && n_rep <= 2 * sms) {
    // at most two replicas per SM: one block in each of the 2 x SMs slots; the
    // 2 SMs - n largest replicas run alone, the others in large/small pairs
    B->grid = 2 * sms;
    B->n_alone = 2 * sms - n_rep;
  }
  // Capture {args upload, work counter and error words reset, persistent kernel,
  // stats and error words download}: one replay reports every replica's error
  // word without a copy per replica.
  cudaStream_t cs = nullptr;
  cudaGraph_t g = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    bhmc_batch_destroy(B);
    return BHMC_ECUDA;
  }
  bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(B->d_args, B->h_args, sizeof(BatchArgs), cudaMemcpyHostToDevice, cs) == cudaSuccess;
  ok = ok && cudaMemsetAsync(B->d_sched, 0, sched_bytes(n_rep), cs) == cudaSuccess;
  ok = ok && cudaMemsetAsync(B->d_errs, 0, sizeof(int) * n_rep, cs) == cudaSuccess;
  cudaError_t le = cudaSuccess;
  if (ok) {
    le = by_p(B->p, [&](auto PC) { return launch_batch<PC.value>(views[0], B->warps, B->d_views, n_rep, B->grid, B->d_args, B->d_stats, cs); });
  }
  ok = ok && le == cudaSuccess;
  ok = ok && cudaMemcpyAsync(B->h_stats, B->d_stats, sizeof(bhmc_mc_stats) * n_rep, cudaMemcpyDeviceToHost,
                             cs) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(B->h_errs, B->d_errs, sizeof(int) * n_rep, cudaMemcpyDeviceToHost, cs) == cudaSuccess;
  const bool ended = cudaStreamEndCapture(cs, &g) == cudaSuccess;
  ok = ok && ended && cudaGraphInstantiate(&B->graph, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (!ok) {
    bhmc_batch_destroy(B);
    return BHMC_ECUDA;
  }
  *out = B;
  return BHMC_OK;
}

bhmc_status bhmc_batch_destroy(bhmc_batch* B) {
  if (!B) return BHMC_EINVAL;
  if (B->stream) cudaStreamSynchronize(B->stream);
  if (B->graph) cudaGraphExecDestroy(B->graph);
  for (bhmc_ctx* c : B->reps) ctx_free(c);
  cudaFree(B->d_views);
  cudaFree(B->d_args);
  cudaFreeHost(B->h_args);
  cudaFree(B->d_seeds);
  cudaFree(B->d_sched);
  cudaFree(B->d_order);
  cudaFree(B->d_stats);
  cudaFreeHost(B->h_stats);
  cudaFree(B->d_errs);
  cudaFreeHost(B->h_errs);
  delete B;
  return BHMC_OK;
}

bhmc_status bhmc_batch_replica(bhmc_batch* B, int32_t r, bhmc_ctx** ctx) {
  if (!B || !ctx || r < 0 || r >= (int32_t)B->reps.size()) return BHMC_EINVAL;
  *ctx = B->reps[r];
  return BHMC_OK;
}

bhmc_status bhmc_batch_radial_counts(bhmc_batch* B, int32_t nbins, double r_lo, double r_hi, int64_t* counts,
                                     double* charge) {
  if (!B) return BHMC_EINVAL;
  return radial_impl(B->reps.data(), (int)B->reps.size(), nbins, r_lo, r_hi, counts, charge);
}

bhmc_status bhmc_batch_set_radial_sampling(bhmc_batch* B, int32_t nbins, double r_lo, double r_hi,
                                           int64_t every) {
  if (!B) return BHMC_EINVAL;
  const int n = (int)B->reps.size();
  std::vector<SysDev> views(n);
  for (int r = 0; r < n; ++r) {
    bhmc_status rc = rdf_setup(B->reps[r], nbins, r_lo, r_hi, every);
    if (rc != BHMC_OK) return rc;
    views[r] = B->reps[r]->S;
  }
  // the batched kernel reads the replicas' device views
  CK(cudaMemcpy(B->d_views, views.data(), sizeof(SysDev) * n, cudaMemcpyHostToDevice));
  return BHMC_OK;
}

bhmc_status bhmc_batch_get_radial_samples(bhmc_batch* B, int64_t* counts, double* charge, int64_t* n_samples) {
  if (!B || !counts || !charge || !n_samples) return BHMC_EINVAL;
  for (size_t r = 0; r < B->reps.size(); ++r) {
    const int nb = B->reps[r]->S.rdf_nbins;
    bhmc_status rc = rdf_read(B->reps[r], counts + r * (size_t)nb, charge + r * (size_t)nb, n_samples + r);
    if (rc != BHMC_OK) return rc;
  }
  return BHMC_OK;
}

}  // extern "C"

// Checks of a batched call and the host copy of its arguments (seeds uploaded).
static bhmc_status batch_prepare(bhmc_batch* B, uint64_t n_moves, double step, const uint64_t* seeds,
                                 uint64_t move0) {
  if (B)
    for (bhmc_ctx* c : B->reps) c->w_stale = true;
  if (!B || !seeds || !(step >= 0.0)) return BHMC_EINVAL;
  const int n = (int)B->reps.size();
  for (bhmc_ctx* c : B->reps) {
    if (c->sticky) return BHMC_ESTATE;
    if (n_moves > 0 && c->S.n_mob < 1) return BHMC_EINVAL;  // no mobile ion to move
  }
  CK(cudaMemcpyAsync(B->d_seeds, seeds, sizeof(unsigned long long) * n, cudaMemcpyHostToDevice, B->stream));
  CK(cudaStreamSynchronize(B->stream));
  B->h_args->n_moves = n_moves;
  B->h_args->move0 = move0;
  B->h_args->step = step;
  B->h_args->seeds = B->d_seeds;
  B->h_args->order = B->d_order;
  B->h_args->recs = nullptr;
  B->h_args->errs = nullptr;
  B->h_args->claimed = B->d_sched;
  B->h_args->cursor = B->d_sched + n;
  B->h_args->head = B->d_sched + n + 1;
  B->h_args->sm_slot = B->d_sched + n + 2;
  B->h_args->sm_head = B->d_sched + n + 2 + BHMC_SM_IDS;
  B->h_args->n_alone = B->n_alone;
  return BHMC_OK;
}

// One replay of the batched graph; per-move records to `records` (host,
// n_rep x n_moves) when it is non-null.
static bhmc_status batch_run(bhmc_batch* B, uint64_t n_moves, double step, const uint64_t* seeds, uint64_t move0,
                             bhmc_mc_stats* stats, bhmc_move_record* records) {
  bhmc_status rc0 = batch_prepare(B, n_moves, step, seeds, move0);
  if (rc0 != BHMC_OK) return rc0;
  const int n = (int)B->reps.size();
  MoveRec* drec = nullptr;
  const size_t nrec = (size_t)n * n_moves;
  if (records && nrec) {
    if (cudaMalloc(&drec, sizeof(MoveRec) * nrec) != cudaSuccess) return BHMC_ENOMEM;
    B->h_args->recs = drec;
  }
  B->h_args->errs = B->d_errs;
  bhmc_status rc = BHMC_OK;
  if (cudaGraphLaunch(B->graph, B->stream) != cudaSuccess || cudaStreamSynchronize(B->stream) != cudaSuccess) {
    for (bhmc_ctx* c : B->reps) c->sticky = BHMC_ECUDA;
    rc = BHMC_ECUDA;
  } else {
    // every replica's error word came back with the replay; a device error
    // latches in its context as the per-context calls do
    for (int r = 0; r < n; ++r) {
      const int e = B->h_errs[r];
      if (e) {
        B->reps[r]->sticky = e;
        if (rc == BHMC_OK) rc = (bhmc_status)e;
      }
    }
  }
  if (rc == BHMC_OK && drec &&
      cudaMemcpy(records, drec, sizeof(MoveRec) * nrec, cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = BHMC_ECUDA;
  B->h_args->recs = nullptr;
  if (drec) cudaFree(drec);
  if (rc != BHMC_OK) return rc;
  if (stats) std::memcpy(stats, B->h_stats, sizeof(bhmc_mc_stats) * n);
  return BHMC_OK;
}

extern "C" {

bhmc_status bhmc_batch_step_mc(bhmc_batch* B, uint64_t n_moves, double step, const uint64_t* seeds,
                               uint64_t move0, bhmc_mc_stats* stats) {
  return batch_run(B, n_moves, step, seeds, move0, stats, nullptr);
}

bhmc_status bhmc_batch_step_mc_records(bhmc_batch* B, uint64_t n_moves, double step, const uint64_t* seeds,
                                       uint64_t move0, bhmc_mc_stats* stats, bhmc_move_record* records) {
  if (!records) return BHMC_EINVAL;
  return batch_run(B, n_moves, step, seeds, move0, stats, records);
}

bhmc_status bhmc_batch_step_mc_spec(bhmc_batch* B, uint64_t n_moves, double step, const uint64_t* seeds,
                                    uint64_t move0, int32_t proposals, bhmc_mc_stats* stats) {
  if (proposals < 1 || proposals > BHMC_MAX_PROPOSALS) return BHMC_EINVAL;
  bhmc_status rc0 = batch_prepare(B, n_moves, step, seeds, move0);
  if (rc0 != BHMC_OK) return rc0;
  const int n = (int)B->reps.size();
  CK(cudaMemcpyAsync(B->d_args, B->h_args, sizeof(BatchArgs), cudaMemcpyHostToDevice, B->stream));
  CK(cudaMemsetAsync(B->d_stats, 0, sizeof(bhmc_mc_stats) * n, B->stream));
  if (n_moves) {
    const cudaError_t e = by_p(B->p, [&](auto PC) {
      return launch_spec_batch<PC.value>(B->reps[0]->S, B->warps, proposals, B->d_views, n, B->d_args, B->d_stats,
                                         B->stream);
    });
    if (e != cudaSuccess) {
      for (bhmc_ctx* c : B->reps) c->sticky = BHMC_ECUDA;
      return BHMC_ECUDA;
    }
  }
  CK(cudaMemcpyAsync(B->h_stats, B->d_stats, sizeof(bhmc_mc_stats) * n, cudaMemcpyDeviceToHost, B->stream));
  bhmc_status rc = BHMC_OK;
  for (bhmc_ctx* c : B->reps) {
    bhmc_status e = sync_err(c);
    if (e != BHMC_OK && rc == BHMC_OK) rc = e;
  }
  if (rc != BHMC_OK) return rc;
  if (stats) std::memcpy(stats, B->h_stats, sizeof(bhmc_mc_stats) * n);
  return BHMC_OK;
}

}  // extern "C"
