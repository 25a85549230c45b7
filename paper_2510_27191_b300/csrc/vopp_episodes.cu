// Episode mode (Alg. 1-3 as printed): sampled episodes grow a belief tree whose preferences
// are backed up by visit counts.
//
// Planning iteration k = 1, 2, ... (D_max = k) samples M root states from the belief
// (Philox purpose 7), then runs the M episodes depth by depth: each samples an action from
// softmax(Psi(b,.)/eta) (purpose 8), simulates G (transition purpose 9, observation
// purpose 10), adds the reward and a visit to action node (b, a), stops when the new state
// is terminal (FilterTerminals) and otherwise moves to the child belief of the observation,
// creating it on first visit (AppendBeliefs; a continuous observation always creates one).
// Leaves aggregate the heuristic; the backup (Alg. 3) then runs d = D_max .. 1: the visit-
// weighted values of the beliefs at depth d feed Q of their parent action nodes
// (Q = C/N + gamma W/N, Q = 0 for an action without visits), and every belief at depth d-1
// applies V_curr = L Psi, Psi <- Psi - V_curr + Q, V = L Psi.
//
// B300 layout: nodes are rows of dense arrays (action nodes b*A + a; for discrete models a
// dense child table [b][a][o], so AppendBeliefs is one compare-and-claim per episode instead
// of a hash lookup).  New nodes of a depth step are numbered by one scan over the episodes in
// episode order, so the tree is the same on every run and node ids equal the oracle's.
// Reward sums, visit counts, heuristic sums and the backup's accumulations are FP64: the
// sampled decisions of later iterations read Psi, and FP64 keeps them away from the
// rounding-order effects of the atomics; the simulation itself is the FP32 model code of the
// plans, and the exponentials and logarithm of the softmax and log-sum-exp are FP32 (terms
// <= 1, sums in [1, A]).
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "vopp.h"
#include "vopp_device.cuh"
#include "vopp_internal.h"

namespace vopp {

constexpr uint32_t kPurposeEpRoot = 7, kPurposeEpAction = 8, kPurposeEpStep = 9,
                   kPurposeEpObs = 10;
constexpr int kClaimBase = 1 << 30;   // claim of a child slot by episode e: e - 2^30 (< -1)

struct EpDesc {
  int kind, A, O, M, Np, cap;
  double eta, gamma, inv_eta;
  float log2g, h_a0, h_b0;
  int h_zero;
  uint32_t key0, key1;
  double lpi[kMaxActions];
  const DevModel *model;
  // root belief
  const float *rx, *ry;
  const int *rs;
  const float *rw;            // linear weights or null
  const float *rlw;           // log weights (agents) or null
  const float *rpf;           // CROWD root people [12][Np]
  double *cdf;                // [Np]
  // episodes
  float *ex, *ey, *epf;       // NAV2D / CROWD robot, CROWD people [12][M]
  int *es, *eb, *alive, *eslot, *ean;
  // tree
  int *parent_an, *depth;
  double *psi, *V, *C, *Ws, *Hs;
  unsigned long long *N, *Nl;
  int *child;
  // counters: [0] nodes, [1] error, [2] first new node of the last step, [3] new nodes
  int *ctr;
  int K;                      // iterations (= maximum depth)
  int2 *ranges;               // [(K+1) * K]: beliefs of depth d created in iteration j
  int *pre, *bsum;            // assignment scratch: prefix within the block, block sums
  int nblk;                   // blocks of the episode kernels
  unsigned long long *steps;
  double *result;             // [2 + 2A]: action, V(root), Q(root)[A], policy[A]
};

struct EpisodeStore {
  char *buf = nullptr;
  size_t cap_bytes = 0;
  EpDesc d{};
  int n_nodes = 0, A = 0;
};

namespace {

// Warp-aggregated atomic adds: the active lanes that target the same index add their values
// in lane order and one lane issues the atomic (many episodes share the shallow nodes).
__device__ __forceinline__ void agg_add(double *base, long long key, double v) {
  const unsigned act = __activemask();
  const unsigned m = __match_any_sync(act, key);
  double tot = 0.0;
  for (unsigned b = m; b; b &= b - 1) tot += __shfl_sync(m, v, __ffs(b) - 1);
  if ((threadIdx.x & 31) == __ffs(m) - 1) atomicAdd(base + key, tot);
}
__device__ __forceinline__ void agg_count(unsigned long long *base, long long key) {
  const unsigned act = __activemask();
  const unsigned m = __match_any_sync(act, key);
  if ((threadIdx.x & 31) == __ffs(m) - 1) atomicAdd(base + key, (unsigned long long)__popc(m));
}

template <class M>
__device__ __forceinline__ typename M::S ep_load(const EpDesc &P, int e) {
  if constexpr (SelfDraw<M>::value) {
    typename M::S s;
    s.x = P.ex[e];
    s.y = P.ey[e];
    for (int q = 0; q < 6; ++q) { s.px[q] = P.epf[(2 * q) * P.M + e]; s.py[q] = P.epf[(2 * q + 1) * P.M + e]; }
    s.f = P.es[e];
    return s;
  } else if constexpr (M::kStochastic) {
    return typename M::S{P.ex[e], P.ey[e]};
  } else {
    return typename M::S{P.es[e]};
  }
}
template <class M>
__device__ __forceinline__ void ep_store(const EpDesc &P, int e, const typename M::S &s) {
  if constexpr (SelfDraw<M>::value) {
    P.ex[e] = s.x;
    P.ey[e] = s.y;
    for (int q = 0; q < 6; ++q) { P.epf[(2 * q) * P.M + e] = s.px[q]; P.epf[(2 * q + 1) * P.M + e] = s.py[q]; }
    P.es[e] = s.f;
  } else if constexpr (M::kStochastic) {
    P.ex[e] = s.x;
    P.ey[e] = s.y;
  } else {
    P.es[e] = s.s;
  }
}
template <class M>
__device__ __forceinline__ typename M::S ep_root(const EpDesc &P, int i) {
  if constexpr (SelfDraw<M>::value) {
    typename M::S s;
    s.x = P.rx[i];
    s.y = P.ry[i];
    for (int q = 0; q < 6; ++q) { s.px[q] = P.rpf[(2 * q) * P.Np + i]; s.py[q] = P.rpf[(2 * q + 1) * P.Np + i]; }
    s.f = P.rs[i];
    return s;
  } else if constexpr (M::kStochastic) {
    return typename M::S{P.rx[i], P.ry[i]};
  } else {
    return typename M::S{P.rs[i]};
  }
}

// Root CDF in FP64 (terminal particles weigh 0) and the root node.  One CTA.
template <class M>
__device__ void ep_prepare(const EpDesc &P, double *part) {
  const int T = blockDim.x, t = threadIdx.x, Np = P.Np;
  const int chunk = (Np + T - 1) / T, b = t * chunk, e = min(Np, b + chunk);
  double mlw = 0.0;
  if (P.rlw) {   // agents: weights exp(lw - max lw)
    float m = -CUDART_INF_F;
    for (int i = t; i < Np; i += T) m = fmaxf(m, P.rlw[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((t & 31) == 0) part[t >> 5] = (double)m;
    __syncthreads();
    if (t == 0) {
      double mm = -CUDART_INF;
      for (int w = 0; w < (T + 31) / 32; ++w) mm = fmax(mm, part[w]);
      part[64] = mm;
    }
    __syncthreads();
    mlw = part[64];
    __syncthreads();
  }
  auto weight = [&](int i) -> double {
    if (M::terminal(ep_root<M>(P, i))) return 0.0;
    if (P.rlw) return exp((double)P.rlw[i] - mlw);
    return P.rw ? (double)P.rw[i] : 1.0;
  };
  double acc = 0.0;
  for (int i = b; i < e; ++i) acc += weight(i);
  part[t] = acc;
  __syncthreads();
  if (t == 0) {
    double run = 0.0;
    for (int k = 0; k < T; ++k) { const double v = part[k]; part[k] = run; run += v; }
    part[T] = run;
  }
  __syncthreads();
  const double tot = part[T];
  double run = part[t];
  for (int i = b; i < e; ++i) { run += weight(i); P.cdf[i] = run / tot; }
  for (int x = t; x < (P.K + 1) * P.K; x += T) P.ranges[x] = make_int2(0, 0);
  __syncthreads();
  if (t == 0) {
    if (!(tot > 0.0)) P.ctr[1] = 2;     // degenerate root
    P.ctr[0] = 1;
    P.ranges[0] = make_int2(0, 1);      // depth 0: the root
    P.parent_an[0] = -1;
    P.depth[0] = 0;
    P.V[0] = 0.0;
    P.Hs[0] = 0.0;
    P.Nl[0] = 0ull;
  }
  for (int a = t; a < P.A; a += T) {
    P.psi[a] = P.eta * P.lpi[a];
    P.C[a] = 0.0;
    P.N[a] = 0ull;
  }
  for (int x = t; x < P.A * P.O; x += T) P.child[x] = -1;
}

__global__ void __launch_bounds__(1024) k_ep_prepare(EpDesc P) {
  __shared__ double part[1025];
  switch (P.kind) {
    case kNav: ep_prepare<NavModel>(P, part); break;
    case kGrid: ep_prepare<GridModel>(P, part); break;
    case kCrowd: ep_prepare<CrowdModel>(P, part); break;
    default: ep_prepare<ToyModel>(P, part); break;
  }
}

// SampleStatesFromBelief: episode e starts from root particle i with u < cdf[i] (first).
template <class M>
__device__ void ep_start(const EpDesc &P, int e, unsigned long long k) {
  const uint4 w = draw(P.key0, P.key1, (uint32_t)e, kPurposeEpRoot, 0, 0, 0, k);
  const double u = (double)u01(w.x);
  int lo = 0, hi = P.Np - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (u < P.cdf[mid]) hi = mid; else lo = mid + 1;
  }
  ep_store<M>(P, e, ep_root<M>(P, lo));
  P.eb[e] = 0;
  P.alive[e] = 1;
}

__global__ void k_ep_start(EpDesc P, unsigned long long k) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= P.M) return;
  switch (P.kind) {
    case kNav: ep_start<NavModel>(P, e, k); break;
    case kGrid: ep_start<GridModel>(P, e, k); break;
    case kCrowd: ep_start<CrowdModel>(P, e, k); break;
    default: ep_start<ToyModel>(P, e, k); break;
  }
}

// One depth step of every live episode (Alg. 2 body).
template <class M>
__device__ void ep_step(const EpDesc &P, int e, int d, unsigned long long k) {
  if (!P.alive[e]) return;
  const int A = P.A, b = P.eb[e];
  // a ~ softmax(Psi(b,.)/eta), inverse CDF in FP64 (first a with u < cumulative)
  // (the softmax runs in FP32 from the FP64 preferences: its error, ~1e-7 of the total, lies
  // far inside the 1e-5 band in which a sampled decision is treated as a tie)
  const double *ps = P.psi + (long long)b * A;
  double zm = -CUDART_INF;
  for (int a = 0; a < A; ++a) zm = fmax(zm, ps[a] * P.inv_eta);
  float z[kMaxActions], sum = 0.f;
  for (int a = 0; a < A; ++a) { z[a] = __expf((float)(ps[a] * P.inv_eta - zm)); sum += z[a]; }
  const uint4 wa = draw(P.key0, P.key1, (uint32_t)e, kPurposeEpAction, (uint32_t)d, 0, 0, k);
  const float u = u01(wa.x), inv = 1.0f / sum;
  int act = A - 1;
  float run = 0.f;
  for (int a = 0; a < A; ++a) {
    run = fmaf(z[a], inv, run);
    if (u < run) { act = a; break; }
  }
  typename M::S s = ep_load<M>(P, e);
  const uint4 ws = draw(P.key0, P.key1, (uint32_t)e, kPurposeEpStep, (uint32_t)d, 0, 0, k);
  // pair-drawn models take words 0,1 of the episode's call (index 0 of the pair); a
  // self-drawing model keys its own calls by the episode
  const int si = SelfDraw<M>::value ? e : 0;
  const float r = step_particle<M>(s, act, ws, si, DrawCtx{P.key0, P.key1, kPurposeEpStep, (uint32_t)d, k},
                                   *P.model);
  const uint4 wo = draw(P.key0, P.key1, (uint32_t)e, kPurposeEpObs, (uint32_t)d, 0, 0, k);
  const typename M::O o = obs_particle<M>(s, act, wo, DrawCtx{P.key0, P.key1, kPurposeEpObs, (uint32_t)d, k},
                                          (uint32_t)e, *P.model);
  const long long an = (long long)b * A + act;
  agg_add(P.C, an, (double)r);
  agg_count(P.N, an);
  agg_count(P.steps, 0);
  ep_store<M>(P, e, s);
  P.ean[e] = (int)an;
  if (M::terminal(s)) {             // FilterTerminals
    P.alive[e] = 0;
    return;
  }
  if constexpr (!M::kStochastic) {  // discrete observation: claim the child slot
    const int slot = (int)(an * P.O + o.o);
    P.eslot[e] = slot;
    if (P.child[slot] < 0) atomicMin(P.child + slot, e - kClaimBase);
  } else {
    P.eslot[e] = -1;                // continuous: every episode adds a belief
  }
}

__global__ void k_ep_step(EpDesc P, int d, unsigned long long k) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= P.M) return;
  switch (P.kind) {
    case kNav: ep_step<NavModel>(P, e, d, k); break;
    case kGrid: ep_step<GridModel>(P, e, d, k); break;
    case kCrowd: ep_step<CrowdModel>(P, e, d, k); break;
    default: ep_step<ToyModel>(P, e, d, k); break;
  }
}

// AppendBeliefs: the new beliefs of a depth step are numbered in episode order by a scan
// over the episodes' creator flags (block prefixes, one CTA over the block sums), then
// published in the child table, and every live episode moves to its child.
__device__ __forceinline__ bool ep_creator(const EpDesc &P, int e) {
  if (e >= P.M || !P.alive[e]) return false;
  return P.O == 0 || P.child[P.eslot[e]] == e - kClaimBase;
}

__global__ void __launch_bounds__(256) k_ep_flags(EpDesc P) {
  __shared__ int wsum[8];
  const int e = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int f = ep_creator(P, e) ? 1 : 0;
  int incl = f;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  int woff = 0;
  for (int w = 0; w < wid; ++w) woff += wsum[w];
  if (e < P.M) P.pre[e] = woff + incl - f;
  if (threadIdx.x == blockDim.x - 1) P.bsum[blockIdx.x] = woff + incl;
}

__global__ void __launch_bounds__(1024) k_ep_scan(EpDesc P, int d, int k) {
  __shared__ int wsum[32];
  __shared__ int s_base, s_total, s_ok;
  const int T = blockDim.x, t = threadIdx.x, nb = P.nblk;
  const int chunk = (nb + T - 1) / T, b = t * chunk, e_end = min(nb, b + chunk);
  int cnt = 0;
  for (int i = b; i < e_end; ++i) cnt += P.bsum[i];
  const int lane = t & 31, wid = t >> 5;
  int incl = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (t == 0) {
    int run = 0;
    for (int w = 0; w < (T + 31) / 32; ++w) { const int v = wsum[w]; wsum[w] = run; run += v; }
    s_total = run;
    s_base = P.ctr[0];
    s_ok = (s_base + run <= P.cap) ? 1 : 0;
    if (!s_ok) P.ctr[1] = 1;       // capacity exceeded
  }
  __syncthreads();
  int run = s_base + wsum[wid] + incl - cnt;
  for (int i = b; i < e_end; ++i) { const int v = P.bsum[i]; P.bsum[i] = run; run += v; }
  if (t == 0 && s_ok) {
    P.ctr[2] = s_base;
    P.ctr[3] = s_total;
    P.ctr[0] = s_base + s_total;
    P.ranges[(d + 1) * P.K + (k - 1)] = make_int2(s_base, s_total);
  } else if (t == 0) {
    P.ctr[2] = s_base;
    P.ctr[3] = 0;
  }
}

__global__ void __launch_bounds__(256) k_ep_publish(EpDesc P, int d) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (P.ctr[1] != 0 || !ep_creator(P, e)) return;
  const int id = P.bsum[blockIdx.x] + P.pre[e];
  P.parent_an[id] = P.ean[e];
  P.depth[id] = d + 1;
  if (P.O > 0) P.child[P.eslot[e]] = id;
  else P.eb[e] = id;
}

__global__ void __launch_bounds__(256) k_ep_advance(EpDesc P) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= P.M || P.ctr[1] != 0 || !P.alive[e]) return;
  P.eb[e] = P.child[P.eslot[e]];
}

// Fields of the beliefs created by the last assign: Psi_0 = eta log pibar, empty action
// nodes, empty child table, empty leaf sums.
__global__ void k_ep_init_nodes(EpDesc P) {
  const int first = P.ctr[2], count = P.ctr[3], A = P.A, AO = P.A * P.O;
  const long long total = (long long)count * (A > AO ? A : AO);
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
       x += (long long)gridDim.x * blockDim.x) {
    const int per = A > AO ? A : AO;
    const int n = first + (int)(x / per), j = (int)(x % per);
    if (j < A) {
      P.psi[(long long)n * A + j] = P.eta * P.lpi[j];
      P.C[(long long)n * A + j] = 0.0;
      P.N[(long long)n * A + j] = 0ull;
    }
    if (j < AO) P.child[(long long)n * AO + j] = -1;
    if (j == 0) { P.V[n] = 0.0; P.Hs[n] = 0.0; P.Nl[n] = 0ull; }
  }
}

// Leaves: ValueHeuristic aggregated per leaf belief.
template <class M>
__device__ void ep_leaf(const EpDesc &P, int e) {
  if (!P.alive[e]) return;
  const float h = M::heuristic(ep_load<M>(P, e), P.log2g, P.h_a0, P.h_b0, P.h_zero != 0);
  agg_add(P.Hs, P.eb[e], (double)h);
  agg_count(P.Nl, P.eb[e]);
}

__global__ void k_ep_leaf(EpDesc P) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= P.M) return;
  switch (P.kind) {
    case kNav: ep_leaf<NavModel>(P, e); break;
    case kGrid: ep_leaf<GridModel>(P, e); break;
    case kCrowd: ep_leaf<CrowdModel>(P, e); break;
    default: ep_leaf<ToyModel>(P, e); break;
  }
}

// Beliefs of depth dep created up to iteration k, as one index space over the ranges.
struct DepthRanges {
  int2 r[kMaxDepth];
  int n, total;
  __device__ DepthRanges(const EpDesc &P, int dep, int k) : n(0), total(0) {
    for (int j = 0; j < k && j < kMaxDepth; ++j) {
      const int2 v = P.ranges[dep * P.K + j];
      if (v.y > 0) { r[n++] = v; total += v.y; }
    }
  }
  __device__ __forceinline__ int node(int x) const {
    for (int j = 0; j < n; ++j) {
      if (x < r[j].y) return r[j].x + x;
      x -= r[j].y;
    }
    return -1;
  }
};

// Ws of the action nodes of the beliefs at depth d-1 back to zero.
__global__ void k_ep_zero_ws(EpDesc P, int d, int k) {
  const DepthRanges R(P, d - 1, k);
  const long long tot = (long long)R.total * P.A;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < tot;
       x += (long long)gridDim.x * blockDim.x) {
    const int n = R.node((int)(x / P.A));
    P.Ws[(long long)n * P.A + (int)(x % P.A)] = 0.0;
  }
}

// W of the action nodes above depth d: sum over their children of visits x V (leaves of
// this iteration, d = D_max, take V = heuristic mean and their leaf visits).
__global__ void k_ep_scatter(EpDesc P, int d, int dmax) {
  const DepthRanges R(P, d, dmax);
  const int A = P.A;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < R.total; x += gridDim.x * blockDim.x) {
    const int n = R.node(x);
    double visits;
    if (d == dmax) {
      visits = (double)P.Nl[n];
      P.V[n] = P.Nl[n] ? P.Hs[n] / visits : 0.0;
    } else {
      visits = 0.0;
      for (int a = 0; a < A; ++a) visits += (double)P.N[(long long)n * A + a];
    }
    agg_add(P.Ws, P.parent_an[n], visits * P.V[n]);
  }
}

// eta log sum_a exp(Psi_a / eta): the shifted terms (each <= 1) are exponentiated and the
// sum (in [1, A]) logged in FP32, the shift kept in FP64 (absolute error ~1e-7 eta, the same
// on every run).
__device__ __forceinline__ double ep_lse(const double *psi, int A, double eta, double inv_eta) {
  double m = -CUDART_INF;
  for (int a = 0; a < A; ++a) m = fmax(m, psi[a] * inv_eta);
  if (!(m > -CUDART_INF)) return -CUDART_INF;
  float s = 0.f;
  for (int a = 0; a < A; ++a) s += __expf((float)(psi[a] * inv_eta - m));
  return eta * (m + (double)__logf(s));
}

// 1 / n for a visit count: FP32 reciprocal refined by one Newton-Raphson step in FP64
// (r <- r (2 - n r) doubles the correct bits, ~1e-14 relative).
__device__ __forceinline__ double ep_recip(unsigned long long cnt) {
  const double n = (double)cnt;
  const double r = (double)__frcp_rn((float)n);
  return r * fma(-n, r, 2.0);
}

// Preference update of every belief at depth d-1 (Alg. 3: Q, V_curr, Psi, V).
__global__ void k_ep_update(EpDesc P, int d, int k) {
  const DepthRanges R(P, d - 1, k);
  const int A = P.A;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < R.total; x += gridDim.x * blockDim.x) {
    const int n = R.node(x);
    double q[kMaxActions];
    for (int a = 0; a < A; ++a) {
      const long long an = (long long)n * A + a;
      const unsigned long long cnt = P.N[an];
      q[a] = cnt ? (P.C[an] + P.gamma * P.Ws[an]) * ep_recip(cnt) : 0.0;
    }
    double *ps = P.psi + (long long)n * A;
    const double vcur = ep_lse(ps, A, P.eta, P.inv_eta);
    for (int a = 0; a < A; ++a) ps[a] = ps[a] - vcur + q[a];
    P.V[n] = ep_lse(ps, A, P.eta, P.inv_eta);
    if (n == 0)
      for (int a = 0; a < A; ++a) P.result[2 + a] = q[a];
  }
}

// Alg. 1 action choice: argmax Psi(root, .) (lowest index on ties), V, policy.
__global__ void k_ep_result(EpDesc P) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int A = P.A;
  int best = 0;
  for (int a = 1; a < A; ++a) if (P.psi[a] > P.psi[best]) best = a;
  P.result[0] = (double)best;
  P.result[1] = P.V[0];
  for (int a = 0; a < A; ++a) P.result[2 + A + a] = exp((P.psi[a] - P.V[0]) / P.eta);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

void free_episode_store(EpisodeStore *s) {
  if (!s) return;
  if (s->buf) cudaFree(s->buf);
  delete s;
}

int run_plan_episodes(vopp_model *m, const EpisodeInputs &in, const vopp_episode_params &p,
                      double budget_s, vopp_plan_result *out, int32_t *depth_reached,
                      int32_t *n_nodes) {
  const vopp_model_desc &desc = model_desc(m);
  const int A = vopp_model_num_actions(m);
  const int kind = desc.kind;
  const int O = kind == kGrid ? 3 : (kind == kToy ? 2 : (kind == kCrowd ? 64 : 0));
  if (!out) return set_error(VOPP_E_INVALID, "vopp_plan_episodes: out is NULL");
  if (in.N < 1 || in.N > VOPP_MAX_PARTICLES) return set_error(VOPP_E_INVALID, "n_particles outside [1, 65536]");
  if (!in.states) return set_error(VOPP_E_INVALID, "root_states is NULL");
  if (p.episodes < 1 || p.episodes > (1 << 24)) return set_error(VOPP_E_INVALID, "episodes outside [1, 2^24]");
  if (p.max_depth < 1 || p.max_depth > VOPP_MAX_DEPTH) return set_error(VOPP_E_INVALID, "max_depth outside [1, 8]");
  if (!(p.eta > 0.f) || !std::isfinite(p.eta)) return set_error(VOPP_E_INVALID, "eta must be > 0");
  if (!(p.gamma > 0.f && p.gamma < 1.f)) return set_error(VOPP_E_INVALID, "gamma must be in (0,1)");
  if (desc.pi_mode == VOPP_PI_NAV_DIST)
    return set_error(VOPP_E_INVALID, "episode mode keeps no particle sets per node: the distance-softmax reference policy is not available");
  const long long K = p.max_depth, M = p.episodes;
  long long cap = p.max_nodes > 0 ? p.max_nodes : M * K * (K + 1) / 2 + 1;
  if (cap > (1ll << 30) / (A > 1 ? A : 1)) return set_error(VOPP_E_INVALID, "node capacity too large");
  if (!(budget_s > 0.0) || !std::isfinite(budget_s)) budget_s = 0.0;   // no time limit

  vopp_ctx *c = model_ctx(m);
  cudaStream_t st = model_stream(m);
  EpisodeStore *&store = ctx_episode_store(c);
  if (!store) store = new (std::nothrow) EpisodeStore;
  if (!store) return set_error(VOPP_E_NOMEM, "episode store");
  // layout of one buffer
  const size_t Np = (size_t)in.N;
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off = align256(off + bytes); return o; };
  const bool nav = kind == kNav, crowd = kind == kCrowd, xy = nav || crowd;
  const size_t o_rx = take(xy ? 4 * Np : 0), o_ry = take(xy ? 4 * Np : 0);
  const size_t o_rs = take(nav ? 0 : 4 * Np), o_rw = take(4 * Np), o_cdf = take(8 * Np);
  const size_t o_rpf = take(crowd ? 48 * Np : 0);
  const size_t o_ex = take(xy ? 4 * M : 0), o_ey = take(xy ? 4 * M : 0), o_es = take(nav ? 0 : 4 * M);
  const size_t o_epf = take(crowd ? 48 * M : 0);
  const size_t o_eb = take(4 * M), o_alive = take(4 * M), o_eslot = take(4 * M), o_ean = take(4 * M);
  const size_t o_par = take(4 * cap), o_dep = take(4 * cap);
  const size_t o_psi = take(8 * cap * A), o_V = take(8 * cap), o_C = take(8 * cap * A);
  const size_t o_Ws = take(8 * cap * A), o_Hs = take(8 * cap), o_N = take(8 * cap * A), o_Nl = take(8 * cap);
  const size_t o_child = take(4 * cap * A * (O > 0 ? O : 1));
  const size_t nblk = (size_t)((M + 255) / 256);
  const size_t o_ranges = take(8 * (size_t)(K + 1) * K), o_pre = take(4 * M), o_bsum = take(4 * nblk);
  const size_t o_ctr = take(64), o_steps = take(8), o_res = take(8 * (2 + 2 * kMaxActions));
  const size_t bytes = off;
  cudaSetDevice(model_device(m));
  if (bytes > store->cap_bytes) {
    if (store->buf) { cudaStreamSynchronize(st); cudaFree(store->buf); }
    store->buf = nullptr;
    store->cap_bytes = 0;
    if (cudaMalloc(&store->buf, bytes) != cudaSuccess) {
      cudaGetLastError();
      return set_error(VOPP_E_NOMEM, "episode-mode buffers do not fit in device memory");
    }
    store->cap_bytes = bytes;
  }
  char *B = store->buf;
  EpDesc &P = store->d;
  std::memset(&P, 0, sizeof P);
  P.kind = kind; P.A = A; P.O = O; P.M = (int)M; P.Np = in.N; P.cap = (int)cap;
  P.eta = p.eta; P.gamma = p.gamma; P.inv_eta = 1.0 / (double)p.eta;
  const double g = p.gamma;
  P.log2g = (float)std::log2(g);
  P.h_a0 = (float)(-1.0 / (1.0 - g));
  P.h_b0 = (float)((kind == kCrowd ? 1000.0 : 100.0) + 1.0 / (1.0 - g));
  P.h_zero = desc.h_zero;
  P.key0 = (uint32_t)p.seed;
  P.key1 = (uint32_t)(p.seed >> 32);
  {
    double w[kMaxActions], s = 0.0;
    for (int a = 0; a < A; ++a) { w[a] = desc.pi_mode == VOPP_PI_FIXED ? desc.pi_fixed[a] : 1.0; s += w[a]; }
    if (!(s > 0.0)) return set_error(VOPP_E_INVALID, "the model's fixed policy sums to 0");
    for (int a = 0; a < A; ++a) P.lpi[a] = w[a] > 0.0 ? std::log(w[a] / s) : -INFINITY;
  }
  P.model = model_device_tables(m);
  auto f = [&](size_t o) { return reinterpret_cast<float *>(B + o); };
  auto i32 = [&](size_t o) { return reinterpret_cast<int *>(B + o); };
  auto f64 = [&](size_t o) { return reinterpret_cast<double *>(B + o); };
  auto u64 = [&](size_t o) { return reinterpret_cast<unsigned long long *>(B + o); };
  const bool dev = in.ptr_flags & VOPP_PTR_DEVICE;
  cudaError_t e = cudaSuccess;
  if (crowd) {   // 15 rows of N words: robot x, y, 12 people coordinates, flags
    const float *w = static_cast<const float *>(in.states);
    if (!dev) {
      e = cudaMemcpyAsync(f(o_rx), in.states, 4 * Np, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(f(o_ry), w + Np, 4 * Np, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(f(o_rpf), w + 2 * Np, 48 * Np, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(i32(o_rs), w + 14 * Np, 4 * Np, cudaMemcpyHostToDevice, st);
      w = nullptr;
    }
    P.rx = w ? w : f(o_rx);
    P.ry = w ? w + Np : f(o_ry);
    P.rpf = w ? w + 2 * Np : f(o_rpf);
    P.rs = w ? reinterpret_cast<const int *>(w + 14 * Np) : i32(o_rs);
  } else if (nav) {
    if (dev) {
      P.rx = static_cast<const float *>(in.states);
      P.ry = P.rx + in.N;
    } else {
      e = cudaMemcpyAsync(f(o_rx), in.states, 8 * Np, cudaMemcpyHostToDevice, st);
      P.rx = f(o_rx);
      P.ry = f(o_rx) + in.N;
      (void)o_ry;
    }
  } else {
    if (dev) P.rs = static_cast<const int *>(in.states);
    else {
      e = cudaMemcpyAsync(i32(o_rs), in.states, 4 * Np, cudaMemcpyHostToDevice, st);
      P.rs = i32(o_rs);
    }
  }
  if (in.log_weights) {
    P.rlw = in.log_weights;
  } else if (in.weights) {
    if (dev) P.rw = in.weights;
    else {
      for (size_t i = 0; i < Np; ++i)
        if (!(in.weights[i] >= 0.f) || !std::isfinite(in.weights[i]))
          return set_error(VOPP_E_INVALID, "root weight invalid");
      if (e == cudaSuccess) e = cudaMemcpyAsync(f(o_rw), in.weights, 4 * Np, cudaMemcpyHostToDevice, st);
      P.rw = f(o_rw);
    }
  }
  P.cdf = f64(o_cdf);
  P.ex = f(o_ex); P.ey = f(o_ey); P.es = i32(o_es); P.epf = f(o_epf);
  P.eb = i32(o_eb); P.alive = i32(o_alive); P.eslot = i32(o_eslot); P.ean = i32(o_ean);
  P.parent_an = i32(o_par); P.depth = i32(o_dep);
  P.psi = f64(o_psi); P.V = f64(o_V); P.C = f64(o_C); P.Ws = f64(o_Ws); P.Hs = f64(o_Hs);
  P.N = u64(o_N); P.Nl = u64(o_Nl); P.child = i32(o_child);
  P.ctr = i32(o_ctr); P.steps = u64(o_steps); P.result = f64(o_res);
  P.K = (int)K;
  P.ranges = reinterpret_cast<int2 *>(B + o_ranges);
  P.pre = i32(o_pre);
  P.bsum = i32(o_bsum);
  P.nblk = (int)nblk;
  if (e == cudaSuccess) e = cudaMemsetAsync(B + o_ctr, 0, 64, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(B + o_steps, 0, 8, st);
  if (e != cudaSuccess) return set_error(VOPP_E_CUDA, cudaGetErrorString(e));

  const unsigned eg = (unsigned)((M + 255) / 256);
  const unsigned ng = 148 * 4;
  k_ep_prepare<<<1, 1024, 0, st>>>(P);
  const auto t0 = std::chrono::steady_clock::now();
  int done = 0, hctr[4] = {0, 0, 0, 0};
  for (int k = 1; k <= (int)K; ++k) {
    k_ep_start<<<eg, 256, 0, st>>>(P, (unsigned long long)k);
    for (int d = 0; d < k; ++d) {
      k_ep_step<<<eg, 256, 0, st>>>(P, d, (unsigned long long)k);
      k_ep_flags<<<eg, 256, 0, st>>>(P);
      k_ep_scan<<<1, 1024, 0, st>>>(P, d, k);
      k_ep_publish<<<eg, 256, 0, st>>>(P, d);
      if (O > 0) k_ep_advance<<<eg, 256, 0, st>>>(P);
      k_ep_init_nodes<<<ng, 256, 0, st>>>(P);
    }
    k_ep_leaf<<<eg, 256, 0, st>>>(P);
    for (int d = k; d >= 1; --d) {
      k_ep_zero_ws<<<ng, 256, 0, st>>>(P, d, k);
      k_ep_scatter<<<ng, 256, 0, st>>>(P, d, k);
      k_ep_update<<<ng, 256, 0, st>>>(P, d, k);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hctr, P.ctr, sizeof hctr, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(VOPP_E_CUDA, cudaGetErrorString(e));
    if (hctr[1] == 2) return set_error(VOPP_E_DEGENERATE, "root weights sum to 0");
    if (hctr[1] == 1) return set_error(VOPP_E_NOMEM, "belief-node capacity exceeded (raise max_nodes)");
    done = k;
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (budget_s > 0.0 && el >= budget_s) break;
  }
  k_ep_result<<<1, 32, 0, st>>>(P);
  double res[2 + 2 * kMaxActions];
  unsigned long long steps = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(res, P.result, sizeof(double) * (2 + 2 * A), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&steps, P.steps, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_error(VOPP_E_CUDA, cudaGetErrorString(e));
  std::memset(out, 0, sizeof *out);
  out->action = (int32_t)res[0];
  out->v_root = res[1];
  for (int a = 0; a < A; ++a) { out->q[a] = res[2 + a]; out->policy[a] = res[2 + A + a]; }
  out->particle_steps = steps;
  out->nodes = (uint64_t)hctr[0];
  store->n_nodes = hctr[0];
  store->A = A;
  if (depth_reached) *depth_reached = done;
  if (n_nodes) *n_nodes = hctr[0];
  return VOPP_OK;
}

int episode_tree_read(vopp_ctx *c, int32_t field, uint64_t offset, uint64_t count, void *dst) {
  EpisodeStore *s = ctx_episode_store(c);
  if (!s || !s->buf || !dst) return set_error(VOPP_E_INVALID, "no episode-mode plan on this context");
  const uint64_t nodes = (uint64_t)s->n_nodes, A = (uint64_t)s->A;
  const void *src = nullptr;
  size_t esz = 8;
  uint64_t len = nodes;
  switch (field) {
    case VOPP_EP_PARENT: src = s->d.parent_an; esz = 4; break;
    case VOPP_EP_DEPTH: src = s->d.depth; esz = 4; break;
    case VOPP_EP_PSI: src = s->d.psi; len = nodes * A; break;
    case VOPP_EP_V: src = s->d.V; break;
    case VOPP_EP_REWARD: src = s->d.C; len = nodes * A; break;
    case VOPP_EP_VISITS: src = s->d.N; len = nodes * A; break;
    default: return set_error(VOPP_E_INVALID, "unknown episode-tree field");
  }
  if (offset > len || count > len - offset) return set_error(VOPP_E_INVALID, "range outside the tree");
  cudaStream_t st = ctx_stream(c);
  cudaError_t e = cudaMemcpyAsync(dst, static_cast<const char *>(src) + offset * esz, count * esz,
                                  cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_error(VOPP_E_CUDA, cudaGetErrorString(e));
  return VOPP_OK;
}

}  // namespace vopp

extern "C" {

VOPP_API int vopp_plan_episodes(vopp_model *model, const void *root_states, const float *root_weights,
                                int32_t n_particles, const vopp_episode_params *params, double budget_s,
                                uint32_t ptr_flags, vopp_plan_result *out, int32_t *depth_reached,
                                int32_t *n_nodes) {
  if (!model || !params) return vopp::set_error(VOPP_E_INVALID, "NULL argument");
  vopp::EpisodeInputs in{root_states, root_weights, nullptr, n_particles, ptr_flags};
  return vopp::run_plan_episodes(model, in, *params, budget_s, out, depth_reached, n_nodes);
}

VOPP_API int vopp_episode_tree_read(vopp_ctx *ctx, int32_t field, uint64_t offset, uint64_t count,
                                    void *dst) {
  if (!ctx) return vopp::set_error(VOPP_E_INVALID, "ctx is NULL");
  return vopp::episode_tree_read(ctx, field, offset, count, dst);
}

}  // extern "C"
