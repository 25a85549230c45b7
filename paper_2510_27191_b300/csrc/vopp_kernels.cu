// vopp_kernels.cu -- the VOPP hot path on sm_103a.
//
// Full-width belief-tree expansion (Alg. 2, full-width form) and the closed-form
// Reference-Based backup (Alg. 3 with one Eq. 3 update, Eq. 1 value):
//   k_root_prep   normalise the root belief, zero terminal particles (Alg. 1 sample step)
//   k_expand      materialise level l+1 children: step every particle of the parent under
//                 (a, k), draw the branch observation, reweight, write the child SoA
//   k_leaf        per level-(D-1) node: build its particle set in shared memory (or load
//                 it), expand all A*W leaf children without writing particles (weighted
//                 heuristic mean, branch weights, mean reward), then back the node up
//                 and climb: the last child of each parent to finish backs the parent up,
//                 up to the FP64 root and the action choice (no separate backup launches)
//   k_belief      SIR belief update tau(b, a, o) of one agent (Sec. III-B)
//
// No tensor cores: nothing here is a dense contraction.  The leaf kernel is bound by FP32
// / SFU issue (Philox integer multiplies, Box-Muller, log / exp); the others are small.
#include <type_traits>

#include "vopp_device.cuh"
#include "vopp_internal.h"
#include "vopp.h"

namespace vopp {

// ---------------------------------------------------------------------------------------
// Programmatic dependent launch: a kernel lets the next kernel of the plan start being
// scheduled right away, and waits for its predecessor's results before reading them.  Both
// are no-ops for a kernel launched without the programmatic-serialisation attribute.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void pdl_release_next() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait_prev() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---------------------------------------------------------------------------------------
// Particle-set views.
//   GNode: a node's particles in a global level store (SoA x[N], y[N] / s[N], lw[N]); the
//          linear weight is exp(lw).
//   SNode: a node's particles in shared memory, pair-interleaved so that one 16-byte load
//          gives both particles of a Philox pair: NAV2D {x0,x1,y0,y1}, TOY2 {s0,s1}, then
//          {lw0,lw1,w0,w1}; GRID {w0,w1} then {s0,s1}.  Odd N pads the last pair with a
//          zero-weight particle.
// ---------------------------------------------------------------------------------------
template <class M> struct GNode;
template <> struct GNode<NavModel> {
  float *x, *y, *lwp;
  __device__ static GNode at(const PlanDesc &P, int l, long long node) {
    const long long b = node * P.N;
    return GNode{P.px[l] + b, P.py[l] + b, P.plw[l] + b};
  }
  __device__ __forceinline__ NavModel::S get(int i) const { return NavModel::S{x[i], y[i]}; }
  __device__ __forceinline__ void put(int i, const NavModel::S &s) const { x[i] = s.x; y[i] = s.y; }
  __device__ __forceinline__ float lw(int i) const { return lwp[i]; }
  __device__ __forceinline__ void set_lw(int i, float v) const { lwp[i] = v; }
};
template <class M> struct GNodeInt {
  int *s;
  float *lwp;
  __device__ static GNodeInt at(const PlanDesc &P, int l, long long node) {
    const long long b = node * P.N;
    return GNodeInt{P.ps[l] + b, P.plw[l] + b};
  }
  __device__ __forceinline__ typename M::S get(int i) const { return typename M::S{s[i]}; }
  __device__ __forceinline__ void put(int i, const typename M::S &v) const { s[i] = v.s; }
  __device__ __forceinline__ float lw(int i) const { return lwp[i]; }
  __device__ __forceinline__ void set_lw(int i, float v) const { lwp[i] = v; }
};
template <> struct GNode<GridModel> : GNodeInt<GridModel> {
  __device__ static GNode at(const PlanDesc &P, int l, long long node) {
    GNode r; static_cast<GNodeInt<GridModel> &>(r) = GNodeInt<GridModel>::at(P, l, node); return r;
  }
};
template <> struct GNode<ToyModel> : GNodeInt<ToyModel> {
  __device__ static GNode at(const PlanDesc &P, int l, long long node) {
    GNode r; static_cast<GNodeInt<ToyModel> &>(r) = GNodeInt<ToyModel>::at(P, l, node); return r;
  }
};

template <> struct GNode<CrowdModel> {
  float *x, *y, *pf, *lwp;
  int *f;
  int N;
  __device__ static GNode at(const PlanDesc &P, int l, long long node) {
    const long long b = node * P.N;
    return GNode{P.px[l] + b, P.py[l] + b, P.pf[l] + 12 * b, P.plw[l] + b, P.ps[l] + b, P.N};
  }
  __device__ __forceinline__ CrowdModel::S get(int i) const {
    CrowdModel::S s;
    s.x = x[i];
    s.y = y[i];
#pragma unroll
    for (int q = 0; q < 6; ++q) { s.px[q] = pf[(2 * q) * N + i]; s.py[q] = pf[(2 * q + 1) * N + i]; }
    s.f = f[i];
    return s;
  }
  __device__ __forceinline__ void put(int i, const CrowdModel::S &s) const {
    x[i] = s.x;
    y[i] = s.y;
#pragma unroll
    for (int q = 0; q < 6; ++q) { pf[(2 * q) * N + i] = s.px[q]; pf[(2 * q + 1) * N + i] = s.py[q]; }
    f[i] = s.f;
  }
  __device__ __forceinline__ float lw(int i) const { return lwp[i]; }
  __device__ __forceinline__ void set_lw(int i, float v) const { lwp[i] = v; }
};

template <class M> struct SNode;
// NAV2D leaf node, pair-interleaved so that one 16-byte load feeds a Philox pair:
// A = (x0, x1, y0, y1) / 16 (positions in units of 16, a power-of-two scaling, so get / put
// convert exactly), B = (lw0, lw1, w0, w1) (base-2 log weights, linear weights), Mk = (m0, m1)
// (1 for a live particle, 0 for a terminal one).
template <> struct SNode<NavModel> {
  float4 *A, *B;
  float2 *Mk;
  static constexpr int kPairBytes = 40;
  __device__ static SNode at(float *base, int npairs) {
    float4 *p = reinterpret_cast<float4 *>(base);
    return SNode{p, p + npairs, reinterpret_cast<float2 *>(p + 2 * npairs)};
  }
  __device__ __forceinline__ NavModel::S get(int i) const {
    const float *a = reinterpret_cast<const float *>(A + (i >> 1));
    return NavModel::S{16.0f * a[i & 1], 16.0f * a[2 + (i & 1)]};
  }
  __device__ __forceinline__ void put(int i, const NavModel::S &s) const {
    float *a = reinterpret_cast<float *>(A + (i >> 1));
    a[i & 1] = 0.0625f * s.x;
    a[2 + (i & 1)] = 0.0625f * s.y;
  }
  __device__ __forceinline__ void get_pair(int p, NavModel::S &s0, NavModel::S &s1) const {
    const float4 a = A[p];
    s0 = NavModel::S{16.0f * a.x, 16.0f * a.z};
    s1 = NavModel::S{16.0f * a.y, 16.0f * a.w};
  }
  __device__ __forceinline__ float4 A16(int p) const { return A[p]; }   // scaled by 1/16
  __device__ __forceinline__ float4 xy(int p) const {                   // unscaled
    const float4 a = A[p];
    return make_float4(16.0f * a.x, 16.0f * a.y, 16.0f * a.z, 16.0f * a.w);
  }
  __device__ __forceinline__ float m(int i) const { return reinterpret_cast<const float *>(Mk + (i >> 1))[i & 1]; }
  __device__ __forceinline__ void set_m(int i, float v) const { reinterpret_cast<float *>(Mk + (i >> 1))[i & 1] = v; }
  __device__ __forceinline__ float lw(int i) const { return reinterpret_cast<const float *>(B + (i >> 1))[i & 1]; }
  __device__ __forceinline__ void set_lw(int i, float v) const { reinterpret_cast<float *>(B + (i >> 1))[i & 1] = v; }
  __device__ __forceinline__ float w(int i) const { return reinterpret_cast<const float *>(B + (i >> 1))[2 + (i & 1)]; }
  __device__ __forceinline__ void set_w(int i, float v) const { reinterpret_cast<float *>(B + (i >> 1))[2 + (i & 1)] = v; }
  __device__ __forceinline__ float4 pairB(int p) const { return B[p]; }   // (lw0, lw1, w0, w1)
};

template <class M> struct SNodeInt {
  int2 *A;
  float4 *B;
  static constexpr int kPairBytes = 24;
  __device__ static SNodeInt at(float *base, int npairs) {
    float4 *b = reinterpret_cast<float4 *>(base);
    return SNodeInt{reinterpret_cast<int2 *>(b + npairs), b};
  }
  __device__ __forceinline__ typename M::S get(int i) const {
    return typename M::S{reinterpret_cast<const int *>(A + (i >> 1))[i & 1]};
  }
  __device__ __forceinline__ void put(int i, const typename M::S &v) const {
    reinterpret_cast<int *>(A + (i >> 1))[i & 1] = v.s;
  }
  __device__ __forceinline__ void get_pair(int p, typename M::S &s0, typename M::S &s1) const {
    const int2 a = A[p];
    s0 = typename M::S{a.x};
    s1 = typename M::S{a.y};
  }
  __device__ __forceinline__ float lw(int i) const { return reinterpret_cast<const float *>(B + (i >> 1))[i & 1]; }
  __device__ __forceinline__ void set_lw(int i, float v) const { reinterpret_cast<float *>(B + (i >> 1))[i & 1] = v; }
  __device__ __forceinline__ float w(int i) const { return reinterpret_cast<const float *>(B + (i >> 1))[2 + (i & 1)]; }
  __device__ __forceinline__ void set_w(int i, float v) const { reinterpret_cast<float *>(B + (i >> 1))[2 + (i & 1)] = v; }
  __device__ __forceinline__ float4 pairB(int p) const { return B[p]; }   // (lw0, lw1, w0, w1)
};
// GRID leaf node: {s0, s1} and {w0, w1} (linear weights) per pair, 16 B, and no stored log
// weights: the rare log-domain path recomputes a particle's base-2 log weight as the node
// build made it, from the per-node values in s_grid_lw -- which leaves shared memory for the
// sense table by (rock, cell).
struct GridLwCtx {
  const float *par_lw;    // leaf_gen: the parent's natural log weights (its level store)
  const float *node_lw;   // otherwise: the node's own natural log weights (its level store)
  const DevModel *dm;
  float lse2;             // the node build's base-2 normaliser
  int a, o, N, gen;       // the node's action and observation, N, leaf_gen
};
__shared__ GridLwCtx s_grid_lw;
template <> struct SNode<GridModel> {
  int2 *A;
  float2 *W2;
  static constexpr int kPairBytes = 16;
  __device__ static SNode at(float *base, int npairs) {
    float2 *w = reinterpret_cast<float2 *>(base);
    return SNode{reinterpret_cast<int2 *>(w + npairs), w};
  }
  __device__ __forceinline__ GridModel::S get(int i) const {
    return GridModel::S{reinterpret_cast<const int *>(A + (i >> 1))[i & 1]};
  }
  __device__ __forceinline__ void put(int i, const GridModel::S &v) const {
    reinterpret_cast<int *>(A + (i >> 1))[i & 1] = v.s;
  }
  __device__ __forceinline__ void get_pair(int p, GridModel::S &s0, GridModel::S &s1) const {
    const int2 a = A[p];
    s0 = GridModel::S{a.x};
    s1 = GridModel::S{a.y};
  }
  __device__ __forceinline__ float w(int i) const { return reinterpret_cast<const float *>(W2 + (i >> 1))[i & 1]; }
  __device__ __forceinline__ void set_w(int i, float v) const { reinterpret_cast<float *>(W2 + (i >> 1))[i & 1] = v; }
  __device__ __forceinline__ void set_lw(int, float) const {}   // not stored (see lw)
  // the node build's value, bit for bit: (lw_parent log2 e + log2 Z) - lse2 with leaf_gen
  // (node_build, pass 3), lw log2 e from a materialised level otherwise; -inf past N
  __device__ __forceinline__ float lw(int i) const {
    const GridLwCtx &c = s_grid_lw;
    if (i >= c.N) return -CUDART_INF_F;
    if (!c.gen) return kLog2e * c.node_lw[i];
    if (!(c.lse2 > -CUDART_INF_F)) return -CUDART_INF_F;
    const float e = GridModel::loglik2(get(i), c.a, GridModel::O{c.o}, *c.dm);
    return fmaf(c.par_lw[i], kLog2e, e) - c.lse2;
  }
  __device__ __forceinline__ float4 pairB(int p) const {
    const float2 w2 = W2[p];
    return make_float4(lw(2 * p), lw(2 * p + 1), w2.x, w2.y);
  }
};
template <> struct SNode<ToyModel> : SNodeInt<ToyModel> {
  __device__ static SNode at(float *base, int np) {
    SNode r; static_cast<SNodeInt<ToyModel> &>(r) = SNodeInt<ToyModel>::at(base, np); return r;
  }
};

// CROWD in shared memory: {lw0,lw1,w0,w1} per pair, then 15 rows of 2*npairs words (robot
// x, y, the 12 people coordinates, the flags).
template <> struct SNode<CrowdModel> {
  float4 *B;
  float *F;
  int n2;
  static constexpr int kPairBytes = 16 + 2 * 15 * 4;
  __device__ static SNode at(float *base, int npairs) {
    float4 *b = reinterpret_cast<float4 *>(base);
    return SNode{b, reinterpret_cast<float *>(b + npairs), 2 * npairs};
  }
  __device__ __forceinline__ CrowdModel::S get(int i) const {
    CrowdModel::S s;
    s.x = F[i];
    s.y = F[n2 + i];
#pragma unroll
    for (int q = 0; q < 6; ++q) { s.px[q] = F[(2 + 2 * q) * n2 + i]; s.py[q] = F[(3 + 2 * q) * n2 + i]; }
    s.f = __float_as_int(F[14 * n2 + i]);
    return s;
  }
  __device__ __forceinline__ void put(int i, const CrowdModel::S &s) const {
    F[i] = s.x;
    F[n2 + i] = s.y;
#pragma unroll
    for (int q = 0; q < 6; ++q) { F[(2 + 2 * q) * n2 + i] = s.px[q]; F[(3 + 2 * q) * n2 + i] = s.py[q]; }
    F[14 * n2 + i] = __int_as_float(s.f);
  }
  __device__ __forceinline__ void get_pair(int p, CrowdModel::S &s0, CrowdModel::S &s1) const {
    s0 = get(2 * p);
    s1 = get(2 * p + 1);
  }
  __device__ __forceinline__ float lw(int i) const { return reinterpret_cast<const float *>(B + (i >> 1))[i & 1]; }
  __device__ __forceinline__ void set_lw(int i, float v) const { reinterpret_cast<float *>(B + (i >> 1))[i & 1] = v; }
  __device__ __forceinline__ float w(int i) const { return reinterpret_cast<const float *>(B + (i >> 1))[2 + (i & 1)]; }
  __device__ __forceinline__ void set_w(int i, float v) const { reinterpret_cast<float *>(B + (i >> 1))[2 + (i & 1)] = v; }
  __device__ __forceinline__ float4 pairB(int p) const { return B[p]; }   // (lw0, lw1, w0, w1)
};

// Scratch for the two per-particle values a child build keeps between its passes.
struct ScratchArrays {           // K2: dynamic shared memory, N floats each
  float *L, *E;
  __device__ __forceinline__ float getL(int i) const { return L[i]; }
  __device__ __forceinline__ void setL(int i, float v) const { L[i] = v; }
  __device__ __forceinline__ float getE(int i) const { return E[i]; }
  __device__ __forceinline__ void setE(int i, float v) const { E[i] = v; }
};
template <class M> struct ScratchInNode {   // K3: the destination node's lw / w slots
  SNode<M> n;
  __device__ __forceinline__ float getL(int i) const { return n.lw(i); }
  __device__ __forceinline__ void setL(int i, float v) const { n.set_lw(i, v); }
  __device__ __forceinline__ float getE(int i) const { return n.w(i); }
  __device__ __forceinline__ void setE(int i, float v) const { n.set_w(i, v); }
};
template <> struct ScratchInNode<GridModel> {   // L in the linear-weight slot, then w there
  SNode<GridModel> n;
  __device__ __forceinline__ float getL(int i) const { return n.w(i); }
  __device__ __forceinline__ void setL(int i, float v) const { n.set_w(i, v); }
  __device__ __forceinline__ float getE(int i) const { return n.w(i); }
  __device__ __forceinline__ void setE(int i, float v) const { n.set_w(i, v); }
};

// A branch observation from its two-float form (obs_f2): NAV2D (x, y); the discrete models'
// index is exact in the first float.
template <class M> __device__ __forceinline__ typename M::O obs_from_f2(float2 f) {
  return typename M::O{(int)f.x};
}
template <> __device__ __forceinline__ NavModel::O obs_from_f2<NavModel>(float2 f) {
  return NavModel::O{f.x, f.y};
}

// The observation of a pair-packed (NAV2D) branch; other models never take that path.
template <class Obs> __device__ __forceinline__ NavModel::O o_nav(const Obs &) { return NavModel::O{0.f, 0.f}; }
template <> __device__ __forceinline__ NavModel::O o_nav<NavModel::O>(const NavModel::O &o) { return o; }

template <class M> __device__ __forceinline__ float2 state_xy(const typename M::S &s);
template <> __device__ __forceinline__ float2 state_xy<NavModel>(const NavModel::S &s) {
  return make_float2(s.x, s.y);
}
template <> __device__ __forceinline__ float2 state_xy<GridModel>(const GridModel::S &) {
  return make_float2(0.f, 0.f);
}
template <> __device__ __forceinline__ float2 state_xy<ToyModel>(const ToyModel::S &) {
  return make_float2(0.f, 0.f);
}
template <> __device__ __forceinline__ float2 state_xy<CrowdModel>(const CrowdModel::S &s) {
  return make_float2(s.x, s.y);
}

template <class M> __device__ __forceinline__ typename M::S set_xy(typename M::S s, float, float) { return s; }
template <> __device__ __forceinline__ NavModel::S set_xy<NavModel>(NavModel::S, float x, float y) {
  return NavModel::S{x, y};
}

template <class M>
__device__ __forceinline__ typename M::S load_root(const PlanDesc &P, int i);
template <> __device__ __forceinline__ NavModel::S load_root<NavModel>(const PlanDesc &P, int i) {
  return NavModel::S{P.root_x[i], P.root_y[i]};
}
template <> __device__ __forceinline__ GridModel::S load_root<GridModel>(const PlanDesc &P, int i) {
  // Host states are checked by the library; a device buffer's out-of-range fields are
  // clamped (x <= 11, y <= 10, bits 17-31 cleared) so that every table index stays in range.
  const int s = P.root_s[i];
  return GridModel::S{(s & 0x100FF) | (min(gx(s), 11) << 8) | (min(gy(s), 10) << 12)};
}
template <> __device__ __forceinline__ ToyModel::S load_root<ToyModel>(const PlanDesc &P, int i) {
  return ToyModel::S{P.root_s[i]};
}
template <> __device__ __forceinline__ CrowdModel::S load_root<CrowdModel>(const PlanDesc &P, int i) {
  CrowdModel::S s;
  s.x = P.root_x[i];
  s.y = P.root_y[i];
#pragma unroll
  for (int q = 0; q < 6; ++q) { s.px[q] = P.root_pf[(2 * q) * P.N + i]; s.py[q] = P.root_pf[(2 * q + 1) * P.N + i]; }
  s.f = P.root_s[i];
  return s;
}

// Transition Philox words of particle pair p of branch (a, k) of the node with key node
// index kn at level l (kn = key_node(P, l, node)).
template <class M>
__device__ __forceinline__ uint4 pair_words(const PlanDesc &P, int p, int l, int a, int k,
                                            unsigned long long kn) {
  if (!M::kStochastic) return make_uint4(0u, 0u, 0u, 0u);
  return draw(P.key0, P.key1, (uint32_t)p, kPurposeTransition, key_level(P, l), a, k, kn);
}

// The branch observation of branch (a, k) of the node with key node index kn at level l:
// enumerated, or drawn from the representative particle j = floor(u N / 2^32) after its
// own transition.
template <class M, class Src>
__device__ __forceinline__ typename M::O branch_obs(const PlanDesc &P, const Src &src, int l, int a,
                                                    int k, unsigned long long kn,
                                                    const DevModel &dm, int &j) {
  if (P.branch_mode == kEnumerate) { j = -1; return M::enum_obs(k); }
  const uint4 w = draw(P.key0, P.key1, 0u, kPurposeObservation, key_level(P, l), a, k, kn);
  j = (int)(((unsigned long long)w.z * (unsigned long long)P.N) >> 32);
  typename M::S sj = src.get(j);
  const uint4 t = pair_words<M>(P, j >> 1, l, a, k, kn);
  const uint32_t c1 = key_level(P, l) | ((uint32_t)a << 8) | ((uint32_t)k << 16);
  step_particle<M>(sj, a, t, j, DrawCtx{P.key0, P.key1, kPurposeTransition, c1, kn}, dm);
  return obs_particle<M>(sj, a, w, DrawCtx{P.key0, P.key1, kPurposeObservation, c1, kn}, 0u, dm);
}

// log pibar(a | node) for a < A (computed by every calling thread).
__device__ __forceinline__ float log_pibar(const PlanDesc &P, float2 mu, int a) {
  if (P.pi_mode != kPiNavDist) return P.log_pi[a];
  float z[4], zm = -CUDART_INF_F;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const float cx = fminf(fmaxf(mu.x + NavModel::dx_of(b), 0.f), 10.f);
    const float cy = fminf(fmaxf(mu.y + NavModel::dy_of(b), 0.f), 10.f);
    z[b] = -sqrtf(cx * cx + cy * cy) / P.pi_temp;
    zm = fmaxf(zm, z[b]);
  }
  float s = 0.f;
#pragma unroll
  for (int b = 0; b < 4; ++b) s += __expf(z[b] - zm);
  float za = z[0];
#pragma unroll
  for (int b = 1; b < 4; ++b) za = (a == b) ? z[b] : za;
  return za - zm - __logf(s);
}

// Philox pairs per thread between two rescales of a child build's running sums (NAV2D 2:
// leaf 254.8 -> 253.6 us; GRID 1: 4.59 -> 4.61 ms at 2 on the depth-4 grid plan).
template <class M> struct BuildChunk { static constexpr int value = 1; };
template <> struct BuildChunk<NavModel> { static constexpr int value = 2; };
// Floats of the block-reduction buffer a child build needs (7 per-warp values, 32 warps).
constexpr int kRedFloats = 32 * 7;

// ---------------------------------------------------------------------------------------
// Child construction (Alg. 2: G, observation, weighting) by a whole CTA, one Philox pair
// per thread iteration, in base-2 logs.  src: parent particles (level l, natural log
// weights); dst: the child's particles; sc: two per-particle scratch values between the
// passes; red: kRedFloats floats of shared memory.  dst_log2: store the child's log weights
// in base 2 (shared-memory node buffers)
// rather than natural (level stores); dst_has_w also stores the linear weights.
// ---------------------------------------------------------------------------------------
template <class M, class Src, class Dst, class Scr>
__device__ void build_child(const PlanDesc &P, const DevModel &dm, int l,
                            unsigned long long child, const Src &src, const Dst &dst,
                            const Scr &sc, float *red, bool dst_has_w, bool dst_log2,
                            float2 *mu_out, typename M::O *o_out = nullptr,
                            float *lse2_out = nullptr) {
  const int N = P.N, AW = P.AW, W = P.W, npairs = (N + 1) >> 1;
  constexpr int kBC = BuildChunk<M>::value;
  const unsigned long long parent = child / (unsigned long long)AW;
  const int slot = (int)(child - parent * (unsigned long long)AW);
  const int a = slot / W, k = slot - (slot / W) * W;
  int j;
  const unsigned long long kn = key_node(P, l, parent);
  const typename M::O o = branch_obs<M>(P, src, l, a, k, kn, dm, j);
  const uint32_t c1 = key_level(P, l) | ((uint32_t)a << 8) | ((uint32_t)k << 16);

  // pass 1: step every particle, log2-likelihood, reward mean; keep L2 = lw2 + ell2 for the
  // normalisation, and fold L2 (child weights, mean particle) and ell2 (the proposal
  // normaliser of omega) into per-thread running max-shifted sums, one rescale per chunk of
  // kBC pairs (then one block-wide merge instead of a second pass and a reduction)
  const bool want_mu = P.pi_mode == kPiNavDist;
  Kahan R, S1, S0, MX, MY;
  R.init(); S1.init(); S0.init(); MX.init(); MY.init();
  float m1 = -CUDART_INF_F, m0 = -CUDART_INF_F;
  // GRID: whole chunks of kBC pairs per thread, when npairs allows, with no bounds test
  // (depth-4 grid leaf 4.35 -> 4.28 ms; the navigation leaf is slower that way)
  auto pass1 = [&](auto full_tag) {
    constexpr bool kFull = decltype(full_tag)::value;
  for (int base = threadIdx.x; base < npairs; base += blockDim.x * kBC) {
    float Lc[2 * kBC], Ec[2 * kBC], Xc[2 * kBC], Yc[2 * kBC];
    float cm1 = -CUDART_INF_F, cm0 = -CUDART_INF_F, rp = 0.f;
#pragma unroll
    for (int c = 0; c < kBC; ++c) {
      const int p = base + c * blockDim.x;
      Lc[2 * c] = Lc[2 * c + 1] = Ec[2 * c] = Ec[2 * c + 1] = -CUDART_INF_F;
      Xc[2 * c] = Xc[2 * c + 1] = Yc[2 * c] = Yc[2 * c + 1] = 0.f;
      if (kFull || p < npairs) {
        const int i0 = 2 * p, i1 = 2 * p + 1;
        const bool v1 = i1 < N;
        const uint4 w = M::kStochastic
                            ? philox(make_uint4(c1, (uint32_t)p, (uint32_t)kn, (uint32_t)(kn >> 32)),
                                     P.key0, P.key1)
                            : make_uint4(0u, 0u, 0u, 0u);
        const float lw0 = src.lw(i0), lw1 = v1 ? src.lw(i1) : -CUDART_INF_F;
        float2 r, e;
        typename M::S s0 = src.get(i0), s1 = v1 ? src.get(i1) : src.get(i0);
        if constexpr (M::kPairPacked) {
          float2 X = make_float2(state_xy<M>(s0).x, state_xy<M>(s1).x);
          float2 Y = make_float2(state_xy<M>(s0).y, state_xy<M>(s1).y);
          bool t0, t1;
          r = NavModel::step_pair(X, Y, NavModel::dx_of(a), NavModel::dy_of(a), w, t0, t1);
          e = NavModel::loglik2_pair(X, Y, o_nav(o));
          s0 = set_xy<M>(s0, X.x, Y.x);
          s1 = set_xy<M>(s1, X.y, Y.y);
        } else {
          const DrawCtx dc{P.key0, P.key1, kPurposeTransition, c1, kn};
          r.x = step_particle<M>(s0, a, w, i0, dc, dm);
          r.y = step_particle<M>(s1, a, w, i1, dc, dm);
          e = make_float2(M::loglik2(s0, a, o, dm), M::loglik2(s1, a, o, dm));
        }
        const float L0 = fmaf(lw0, kLog2e, e.x), L1 = v1 ? fmaf(lw1, kLog2e, e.y) : -CUDART_INF_F;
        const float E1 = v1 ? e.y : -CUDART_INF_F;
        if (lw0 > -CUDART_INF_F) rp = fmaf(ex2(lw0 * kLog2e), r.x, rp);
        if (lw1 > -CUDART_INF_F) rp = fmaf(ex2(lw1 * kLog2e), r.y, rp);
        dst.put(i0, s0);
        sc.setL(i0, L0);
        if (v1) {
          dst.put(i1, s1);
          sc.setL(i1, L1);
        }
        Lc[2 * c] = L0;
        Lc[2 * c + 1] = L1;
        Ec[2 * c] = e.x;
        Ec[2 * c + 1] = E1;
        if (want_mu) {
          const float2 q0 = state_xy<M>(s0), q1 = state_xy<M>(s1);
          Xc[2 * c] = q0.x; Yc[2 * c] = q0.y;
          Xc[2 * c + 1] = q1.x; Yc[2 * c + 1] = q1.y;
        }
        cm1 = fmax3(cm1, L0, L1);
        cm0 = fmax3(cm0, e.x, E1);
      }
    }
    // move the shifts to the chunk's maxima, then add the chunk's shifted terms
    if (cm1 > m1) {
      const float f = (m1 > -CUDART_INF_F) ? ex2(m1 - cm1) : 0.f;
      S1.scale(f); MX.scale(f); MY.scale(f);
      m1 = cm1;
    }
    if (cm0 > m0) {
      const float f = (m0 > -CUDART_INF_F) ? ex2(m0 - cm0) : 0.f;
      S0.scale(f);
      m0 = cm0;
    }
    float a1 = 0.f, a0 = 0.f, ax = 0.f, ay = 0.f;
    if (m1 > -CUDART_INF_F) {
#pragma unroll
      for (int t = 0; t < 2 * kBC; ++t) {
        const float x1 = ex2(Lc[t] - m1);   // L = -inf gives 0
        a1 += x1;
        ax = fmaf(x1, Xc[t], ax);
        ay = fmaf(x1, Yc[t], ay);
      }
    }
    if (m0 > -CUDART_INF_F) {
#pragma unroll
      for (int t = 0; t < 2 * kBC; ++t) a0 += ex2(Ec[t] - m0);
    }
    S1.add(a1); S0.add(a0); R.add(rp);
    if (want_mu) { MX.add(ax); MY.add(ay); }
  }
  };
  if (std::is_same<M, GridModel>::value && npairs % (blockDim.x * kBC) == 0) pass1(std::true_type{});
  else pass1(std::false_type{});
  // block-wide merge: each warp merges its lanes' shifted sums at the warp's largest shift,
  // then every warp merges the warps' partial sums the same way (identically in every warp)
  float v[5];
  {
    float w1 = m1, w0 = m0, sv1 = S1.value(), sx = MX.value(), sy = MY.value(), sv0 = S0.value();
    warp_lse2(w1, sv1, sx);
    float dummy = 0.f;
    warp_lse2(w0, sv0, dummy);
    sy *= (m1 > -CUDART_INF_F) ? ex2(m1 - w1) : 0.f;    // MY in the warp's S1 frame
    sy = warp_sum(sy);
    const float rw = warp_sum(R.value());
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();                                    // red may still be read by a caller
    if (lane == 0) {
      red[wid] = w1; red[32 + wid] = sv1; red[64 + wid] = sx; red[96 + wid] = sy;
      red[128 + wid] = w0; red[160 + wid] = sv0; red[192 + wid] = rw;
    }
    __syncthreads();
    float b1 = -CUDART_INF_F, bs1 = 0.f, bx = 0.f, by = 0.f, b0 = -CUDART_INF_F, bs0 = 0.f, br = 0.f;
    if (lane < nw) {
      b1 = red[lane]; bs1 = red[32 + lane]; bx = red[64 + lane]; by = red[96 + lane];
      b0 = red[128 + lane]; bs0 = red[160 + lane]; br = red[192 + lane];
    }
    const float b1_own = b1;
    warp_lse2(b1, bs1, bx);
    by *= (b1_own > -CUDART_INF_F) ? ex2(b1_own - b1) : 0.f;
    by = warp_sum(by);
    float dummy2 = 0.f;
    warp_lse2(b0, bs0, dummy2);
    br = warp_sum(br);
    m1 = b1;
    m0 = b0;
    v[0] = br; v[1] = bs1; v[2] = bs0; v[3] = bx; v[4] = by;
    __syncthreads();                                    // red is free again
  }
  const float rbar = v[0], s1 = v[1], s0 = v[2], mx = v[3], my = v[4];
  const float lse2 = (s1 > 0.f) ? m1 + lg2(s1) : -CUDART_INF_F;       // base 2
  float lom;
  if (P.branch_mode == kEnumerate) lom = kLn2 * lse2;
  else lom = (lse2 > -CUDART_INF_F) ? __logf((float)N) + kLn2 * (lse2 - (m0 + lg2(s0))) : -CUDART_INF_F;

  // pass 3: normalised child log weights (and linear weights)
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const float nl2 = (lse2 > -CUDART_INF_F) ? sc.getL(i) - lse2 : -CUDART_INF_F;
    dst.set_lw(i, dst_log2 ? nl2 : kLn2 * nl2);
    if (dst_has_w) sc.setE(i, ex2(nl2));
    if constexpr (std::is_same<Dst, SNode<NavModel>>::value)   // the leaf's live mask
      dst.set_m(i, NavModel::terminal(dst.get(i)) ? 0.0f : 1.0f);
  }
  const int cl = l + 1;
  if (threadIdx.x == 0) {
    if (cl <= P.D - 2) P.cnt[cl][child] = 0u;   // completion counter of the new node
    P.rbar[cl][child] = rbar;
    P.lom[cl][child] = lom;
    float2 mu = make_float2(0.f, 0.f);
    if (s1 > 0.f) mu = make_float2(mx / s1, my / s1);
    if (P.pi_mode == kPiNavDist && P.mu[cl]) {
      P.mu[cl][2 * child] = mu.x;
      P.mu[cl][2 * child + 1] = mu.y;
    }
    if (mu_out) *mu_out = mu;
    if (o_out) *o_out = o;
    if (lse2_out) *lse2_out = lse2;
    if (P.rep[cl]) P.rep[cl][child] = j;
    if (P.obs[cl]) {   // full detail, or the level-1 observations a kept tree needs
      const float2 of = M::obs_f2(o);
      P.obs[cl][2 * child] = of.x;
      P.obs[cl][2 * child + 1] = of.y;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------
// Backup of one node (Alg. 3: mean reward R, weighted child value W, Q = R + gamma W, then
// the Eq. 1 value over actions) from branch stats held in arrays indexed by slot a*W + k.
// Executed by the lanes of one warp (lane = action).  kL2: the arrays are in global memory
// and written by other CTAs of the running kernel, so they are read through L2 (L1 is not
// coherent across SMs).  Returns V to every lane; lane a's Q in q_lane.
// ---------------------------------------------------------------------------------------
template <bool kL2>
__device__ __forceinline__ float ld_stat(const float *p) {
  if constexpr (kL2) return __ldcg(p);
  else return *p;
}

template <bool kL2>
__device__ __forceinline__ float node_backup_warp(const PlanDesc &P, const float *rb,
                                                  const float *lo, const float *vc, float2 mu,
                                                  float &q_lane, float *psi_node = nullptr,
                                                  bool fresh = false, float *psi_lane = nullptr) {
  const int lane = threadIdx.x & 31, A = P.A, W = P.W;
  float q = 0.f, z = -CUDART_INF_F;
  if (lane < A) {
    float rs = 0.f, M = -CUDART_INF_F;
    // through L2 (a climbing backup, on the plan's critical path at its end) with W <= 4: the
    // three statistics of every branch in one round of loads (navigation leaf 251.8 ->
    // 250.5 us; in shared memory, or for every W, the register arrays cost more than they save)
    constexpr int kWMax = 4;
    float lov[kWMax], vcv[kWMax];
    const bool one = kL2 && W <= kWMax;
    if (one) {
#pragma unroll
      for (int k = 0; k < kWMax; ++k) {
        if (k < W) {
          rs += ld_stat<kL2>(rb + lane * W + k);
          lov[k] = ld_stat<kL2>(lo + lane * W + k);
          vcv[k] = ld_stat<kL2>(vc + lane * W + k);
          M = fmaxf(M, lov[k]);
        }
      }
    } else {
      for (int k = 0; k < W; ++k) {
        rs += ld_stat<kL2>(rb + lane * W + k);
        M = fmaxf(M, ld_stat<kL2>(lo + lane * W + k));
      }
    }
    float fut = 0.f;
    if (M > -CUDART_INF_F) {
      Kahan num, den;
      num.init(); den.init();
      if (one) {
#pragma unroll
        for (int k = 0; k < kWMax; ++k) {
          if (k < W) {
            const float om = __expf(lov[k] - M);
            num.add(om * vcv[k]);
            den.add(om);
          }
        }
      } else {
        for (int k = 0; k < W; ++k) {
          const float om = __expf(ld_stat<kL2>(lo + lane * W + k) - M);
          num.add(om * ld_stat<kL2>(vc + lane * W + k));
          den.add(om);
        }
      }
      fut = num.value() / den.value();
    } else {
      atomicAdd(&P.result->degenerate, 1u);
    }
    q = rs / (float)W + P.gamma * fut;
    if (!psi_node) z = log_pibar(P, mu, lane) + q * P.inv_eta;
  }
  q_lane = q;
  if (psi_node) {
    // Eq. 3 on persistent preferences: V_curr = L Psi, Psi <- Psi - V_curr + Q, V = L Psi
    // (a new node starts from Psi_0 = eta log pibar)
    float ps = -CUDART_INF_F;
    if (lane < A) ps = fresh ? P.eta * log_pibar(P, mu, lane) : psi_node[lane];
    const float zc = ps * P.inv_eta;
    const float zcm = warp_max(zc);
    const float ec = warp_sum((lane < A && zc > -CUDART_INF_F) ? __expf(zc - zcm) : 0.f);
    const float vcur = P.eta * (zcm + __logf(ec));
    const float pn = ps - vcur + q;          // -inf (pibar = 0) stays -inf
    if (lane < A) psi_node[lane] = pn;
    if (psi_lane) *psi_lane = pn;
    z = (lane < A) ? pn * P.inv_eta : -CUDART_INF_F;
  }
  const float zm = warp_max(z);
  float e = (lane < A && z > -CUDART_INF_F) ? __expf(z - zm) : 0.f;
  e = warp_sum(e);
  return P.eta * (zm + __logf(e));
}

// Root backup from the level-1 branch stats and the Alg. 1 action choice (argmax of
// Q + eta log pibar, lowest index on ties), in FP32 with compensated sums; the FP64 variant
// below runs instead when the plan asks for it.  One warp.
__device__ void root_backup_warp_fp64(const PlanDesc &P);
__device__ void root_backup_warp(const PlanDesc &P) {
  if (P.fp64_root) { root_backup_warp_fp64(P); return; }
  const int lane = threadIdx.x & 31, A = P.A;
  float2 mu = make_float2(0.f, 0.f);
  if (P.pi_mode == kPiNavDist) mu = make_float2(__ldcg(P.mu[0]), __ldcg(P.mu[0] + 1));
  float q, ps = -CUDART_INF_F;
  const float v = node_backup_warp<true>(P, P.rbar[1], P.lom[1], P.V[1], mu, q, P.psi[0],
                                         P.psi_new_level <= 0, &ps);
  const float lp = (lane < A) ? log_pibar(P, mu, lane) : -CUDART_INF_F;
  // Alg. 1: the action maximising Psi (closed form: Q + eta log pibar)
  float sc = (lane < A) ? (P.psi[0] ? ps : q + P.eta * lp) : -CUDART_INF_F;
  int best = (lane < A) ? lane : 1 << 30;
  for (int o = 16; o > 0; o >>= 1) {
    const float sc2 = __shfl_xor_sync(0xffffffffu, sc, o);
    const int b2 = __shfl_xor_sync(0xffffffffu, best, o);
    if (sc2 > sc || (sc2 == sc && b2 < best)) { sc = sc2; best = b2; }
  }
  DevResult *R = P.result;
  if (lane < A) {
    R->q[lane] = q;
    R->policy[lane] = P.psi[0] ? __expf((ps - v) * P.inv_eta) : __expf(lp + (q - v) * P.inv_eta);
    P.Q[0][lane] = q;
  }
  if (lane == 0) {
    R->v_root = v;
    R->action = best;
    P.V[0][0] = v;
  }
}

__device__ void root_backup_warp_fp64(const PlanDesc &P) {
  const int lane = threadIdx.x & 31, A = P.A, W = P.W;
  double q = 0.0, z = -CUDART_INF;
  float2 mu = make_float2(0.f, 0.f);
  if (P.pi_mode == kPiNavDist) mu = make_float2(__ldcg(P.mu[0]), __ldcg(P.mu[0] + 1));
  double lp = -CUDART_INF;
  if (lane < A) {
    double rs = 0.0;
    float M = -CUDART_INF_F;
    for (int k = 0; k < W; ++k) {
      rs += (double)__ldcg(P.rbar[1] + lane * W + k);
      M = fmaxf(M, __ldcg(P.lom[1] + lane * W + k));
    }
    double fut = 0.0;
    if (M > -CUDART_INF_F) {
      double num = 0.0, den = 0.0;
      for (int k = 0; k < W; ++k) {
        const double om = exp((double)__ldcg(P.lom[1] + lane * W + k) - (double)M);
        num += om * (double)__ldcg(P.V[1] + lane * W + k);
        den += om;
      }
      fut = num / den;
    } else {
      atomicAdd(&P.result->degenerate, 1u);
    }
    q = rs / (double)W + (double)P.gamma * fut;
    lp = (double)log_pibar(P, mu, lane);
    z = lp + q / (double)P.eta;
  }
  auto lse = [&](double x) {     // eta * log sum over the warp's lanes of exp(x), x = Psi/eta
    double xm = x;
    for (int o = 16; o > 0; o >>= 1) xm = fmax(xm, __shfl_xor_sync(0xffffffffu, xm, o));
    double ex = (lane < A && x > -CUDART_INF) ? exp(x - xm) : 0.0;
    for (int o = 16; o > 0; o >>= 1) ex += __shfl_xor_sync(0xffffffffu, ex, o);
    return (double)P.eta * (xm + log(ex));
  };
  double ps = -CUDART_INF;
  if (P.psi[0]) {   // Eq. 3 on the persistent root preferences
    if (lane < A)
      ps = (P.psi_new_level <= 0) ? (double)P.eta * lp : (double)P.psi[0][lane];
    const double vcur = lse((lane < A) ? ps / (double)P.eta : -CUDART_INF);
    if (lane < A) {
      ps = ps - vcur + q;
      P.psi[0][lane] = (float)ps;
    }
    z = (lane < A) ? ps / (double)P.eta : -CUDART_INF;
  }
  const double v = lse(z);
  double sc = (lane < A) ? (P.psi[0] ? ps : q + (double)P.eta * lp) : -CUDART_INF;
  int best = (lane < A) ? lane : 1 << 30;
  for (int o = 16; o > 0; o >>= 1) {
    const double sc2 = __shfl_xor_sync(0xffffffffu, sc, o);
    const int b2 = __shfl_xor_sync(0xffffffffu, best, o);
    if (sc2 > sc || (sc2 == sc && b2 < best)) { sc = sc2; best = b2; }
  }
  DevResult *R = P.result;
  if (lane < A) {
    R->q[lane] = q;
    R->policy[lane] = P.psi[0] ? exp((ps - v) / (double)P.eta) : exp(lp + (q - v) / (double)P.eta);
    P.Q[0][lane] = (float)q;
  }
  if (lane == 0) {
    R->v_root = v;
    R->action = best;
    R->flags |= 2u;
    P.V[0][0] = (float)v;
  }
}

// After node `node` of level l has its Q and V written: the warp signals the parent, and if
// it is the last of the parent's A*W children to finish, backs the parent up and climbs on.
// The CTA that finishes last overall backs up the root.  Everything a parent's backup reads
// from a child -- its mean reward and branch weight (written by thread 0 of the CTA that built
// it) and its value (lane 0 of the warp that backed it up) -- is written by the lane that
// signals, so its acquire-release atomic on the parent's counter publishes them (release), and
// the last sibling's lane 0 acquires the others' writes before the warp reads them (the warp
// synchronisations order the other lanes after lane 0).  Against a full fence before and after
// the atomic: navigation leaf 254.7 -> 253.1 us.
__device__ __forceinline__ unsigned int atom_add_acq_rel(unsigned int *p) {
  unsigned int old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(p) : "memory");
  return old;
}
__device__ void climb_warp(const PlanDesc &P, int l, unsigned long long node) {
  const int lane = threadIdx.x & 31, A = P.A;
  const unsigned long long AW = (unsigned long long)P.AW;
  unsigned long long n = node;
  for (int lev = l; lev > 0; --lev) {
    __syncwarp();
    const unsigned long long p = n / AW;
    unsigned int old = 0;
    if (lane == 0) old = atom_add_acq_rel(P.cnt[lev - 1] + p);
    old = __shfl_sync(0xffffffffu, old, 0);
    if ((old + 1u) % (unsigned int)AW != 0u) return;
    if (lev - 1 == 0) {
      root_backup_warp(P);
      return;
    }
    const unsigned long long c0 = p * AW;
    float2 mu = make_float2(0.f, 0.f);
    if (P.pi_mode == kPiNavDist) mu = make_float2(__ldcg(P.mu[lev - 1] + 2 * p), __ldcg(P.mu[lev - 1] + 2 * p + 1));
    float q;
    float *psi = P.psi[lev - 1] ? P.psi[lev - 1] + p * A : nullptr;
    const float v = node_backup_warp<true>(P, P.rbar[lev] + c0, P.lom[lev] + c0, P.V[lev] + c0, mu, q,
                                           psi, lev - 1 >= P.psi_new_level);
    if (lane < A) P.Q[lev - 1][p * A + lane] = q;
    if (lane == 0) P.V[lev - 1][p] = v;
    n = p;
  }
}

// ---------------------------------------------------------------------------------------
// K1: root preparation (one CTA per plan).
// ---------------------------------------------------------------------------------------
// Copies in 64 KB slices.
constexpr unsigned long long kCopySlice = 64 * 1024;

// All of one copy by the whole CTA (a plan's level-0 copies in its root preparation CTA).
__device__ __forceinline__ void copy_cta(void *dst, const void *src, unsigned long long bytes) {
  char *d = static_cast<char *>(dst);
  const char *sp = static_cast<const char *>(src);
  const bool v16 = ((reinterpret_cast<uintptr_t>(d) | reinterpret_cast<uintptr_t>(sp) | bytes) & 15) == 0;
  if (v16) {
    uint4 *d4 = reinterpret_cast<uint4 *>(d);
    const uint4 *s4 = reinterpret_cast<const uint4 *>(sp);
    for (unsigned long long w = threadIdx.x; w < bytes / 16; w += blockDim.x)
      d4[w] = sp ? s4[w] : make_uint4(0u, 0u, 0u, 0u);
  } else {
    uint32_t *d1 = reinterpret_cast<uint32_t *>(d);
    const uint32_t *s1 = reinterpret_cast<const uint32_t *>(sp);
    for (unsigned long long w = threadIdx.x; w < bytes / 4; w += blockDim.x) d1[w] = sp ? s1[w] : 0u;
  }
}

// Slice r (in copy-major order, `slices` per copy) of a CopyDesc table, by the whole CTA.
__device__ __forceinline__ void copy_table_slice(const CopyDesc *t, int n, unsigned slices, unsigned r) {
  const unsigned q = r / slices, sl = r - q * slices;
  if (q >= (unsigned)n) return;
  const unsigned long long lo = (unsigned long long)sl * kCopySlice;
  if (lo >= t[q].bytes) return;
  const unsigned long long len = min(t[q].bytes - lo, kCopySlice);
  copy_cta(static_cast<char *>(t[q].dst) + lo, t[q].src ? static_cast<const char *>(t[q].src) + lo : nullptr, len);
}

// The work-item grid of a launch with a copy tail; blocks past it run their slice and
// report true (the caller returns).
__device__ __forceinline__ bool copy_tail_block(const StageTable &st, unsigned &work_grid) {
  work_grid = st.copies ? st.work_grid : gridDim.x;
  if (blockIdx.x < work_grid) return false;
  copy_table_slice(static_cast<const CopyDesc *>(st.copies), st.n_copies, st.copy_slices,
                   blockIdx.x - work_grid);
  return true;
}

template <class M>
__device__ void root_prepare(const PlanDesc &P, const DevModel &dm, const GNode<M> &dst, float *red,
                             bool outputs) {
  const int N = P.N;
  // log weights of the caller's belief; terminal particles and non-positive weights -> -inf.
  // A reused root (a node of a kept tree) is taken as it stands: its particles and
  // normalised log weights are already in the level-0 store, terminal particles included
  // (they keep the weight they had inside that tree, where they add no reward or value).
  float m = -CUDART_INF_F;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    if (P.reuse_root) {
      m = fmaxf(m, dst.lw(i));
      continue;
    }
    const typename M::S s = load_root<M>(P, i);
    float lw;
    if (P.root_lw) {
      lw = P.root_lw[i];
    } else {
      const float w = P.root_w ? P.root_w[i] : 1.0f;
      lw = (w > 0.f) ? logf(w) : -CUDART_INF_F;
    }
    if (!(lw > -CUDART_INF_F) || M::terminal(s)) lw = -CUDART_INF_F;
    dst.put(i, s);
    dst.set_lw(i, lw);
    m = fmaxf(m, lw);
  }
  m = block_max(m, red);
  if (!(m > -CUDART_INF_F)) {
    if (threadIdx.x == 0 && outputs) P.result->status |= kStatusDegenerateRoot;
    return;
  }
  // one pass for the normaliser and the (unnormalised) weighted means of the position and
  // (depth 0) the heuristic, one block reduction for the four sums
  Kahan T, MX, MY, H;
  T.init(); MX.init(); MY.init(); H.init();
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const float lw = dst.lw(i);
    if (!(lw > -CUDART_INF_F)) continue;
    const float e = __expf(lw - m);
    const typename M::S s = dst.get(i);
    const float2 xy = state_xy<M>(s);
    T.add(e);
    MX.add(e * xy.x);
    MY.add(e * xy.y);
    if (P.D == 0) H.add(e * M::heuristic(s, P));
  }
  float sums[4] = {T.value(), MX.value(), MY.value(), H.value()};
  block_sum4(sums, red);
  const float tsum = sums[0];
  const float mx = sums[1] / tsum, my = sums[2] / tsum, hv = sums[3] / tsum;
  if (!P.reuse_root) {   // normalised log weights (a reused root's are already)
    const float lse = m + logf(tsum);
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const float lw = dst.lw(i);
      if (lw > -CUDART_INF_F) dst.set_lw(i, lw - lse);
    }
  }
  if (threadIdx.x == 0 && outputs) {
    if (P.D >= 2) P.cnt[0][0] = 0u;
    if (P.mu[0]) { P.mu[0][0] = mx; P.mu[0][1] = my; }
    if (P.D == 0) {
      // depth 0: V = weighted mean heuristic, every Q equal to it, action = argmax pibar
      DevResult *R = P.result;
      R->v_root = hv;
      int best = 0;
      float bl = -CUDART_INF_F;
      for (int a = 0; a < P.A; ++a) {
        const float lp = log_pibar(P, make_float2(mx, my), a);
        R->q[a] = hv;
        R->policy[a] = exp((double)lp);
        if (lp > bl) { bl = lp; best = a; }
        P.Q[0][a] = hv;
      }
      R->action = best;
      P.V[0][0] = hv;
    }
  }
}

template <class M>
__device__ void root_prep_plan(const PlanDesc &P, const DevModel &dm, float *red) {
  root_prepare<M>(P, dm, GNode<M>::at(P, 0, 0), red, true);
}

__global__ void __launch_bounds__(1024) k_root_prep(const PlanDesc *plans, StageTable st) {
  __shared__ float red[128];
  pdl_release_next();
  const PlanDesc &P = plans[st.plan[blockIdx.x]];
  const DevModel &dm = *P.model;
  switch (P.kind) {
    case kNav: root_prep_plan<NavModel>(P, dm, red); break;
    case kGrid: root_prep_plan<GridModel>(P, dm, red); break;
    case kCrowd: root_prep_plan<CrowdModel>(P, dm, red); break;
    default: root_prep_plan<ToyModel>(P, dm, red); break;
  }
}

// ---------------------------------------------------------------------------------------
// K2: materialise children at level l+1 (one CTA per child).
// ---------------------------------------------------------------------------------------
template <class M>
__device__ void expand_item(const PlanDesc &P, int l, unsigned long long child, float *smem,
                            float *red) {
  const DevModel &dm = *P.model;
  const unsigned long long parent = child / (unsigned long long)P.AW;
  const GNode<M> src = GNode<M>::at(P, l, (long long)parent);
  const GNode<M> dst = GNode<M>::at(P, l + 1, (long long)child);
  const ScratchArrays sc{smem, smem + P.N};
  build_child<M>(P, dm, l, child, src, dst, sc, red, false, false, nullptr);
}

// A node's particles laid out like a level store (GNode) in shared memory from `b`: NAV2D
// x, y, lw; GRID / TOY2 s, lw; CROWD x, y, the people [12][N], lw, flags (root_node_words(kind)
// 32-bit words per particle).
template <class M> __device__ GNode<M> smem_node(float *b, int N);
template <> __device__ GNode<NavModel> smem_node<NavModel>(float *b, int N) {
  return GNode<NavModel>{b, b + N, b + 2 * N};
}
template <> __device__ GNode<GridModel> smem_node<GridModel>(float *b, int N) {
  GNode<GridModel> r;
  r.s = reinterpret_cast<int *>(b);
  r.lwp = b + N;
  return r;
}
template <> __device__ GNode<ToyModel> smem_node<ToyModel>(float *b, int N) {
  GNode<ToyModel> r;
  r.s = reinterpret_cast<int *>(b);
  r.lwp = b + N;
  return r;
}
template <> __device__ GNode<CrowdModel> smem_node<CrowdModel>(float *b, int N) {
  return GNode<CrowdModel>{b, b + N, b + 2 * N, b + 14 * N, reinterpret_cast<int *>(b + 15 * N), N};
}

// A level-1 child of a plan whose root preparation rides in this stage: the CTA prepares
// the root itself into shared memory (every child's CTA does, so no launch waits for a
// separate root kernel), the CTA of child 0 also writes the level-0 store and the root's
// outputs, and the child is built from the shared-memory root.
template <class M>
__device__ void expand_root_item(const PlanDesc &P, unsigned long long child, float *smem,
                                 float *red) {
  const DevModel &dm = *P.model;
  const int N = P.N;
  const GNode<M> root = smem_node<M>(smem + 2 * N, N);
  const bool first = child == 0;
  root_prepare<M>(P, dm, root, red, first);
  __syncthreads();
  if (first) {
    const GNode<M> g = GNode<M>::at(P, 0, 0);
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      g.put(i, root.get(i));
      g.set_lw(i, root.lw(i));
    }
  }
  const GNode<M> dst = GNode<M>::at(P, 1, (long long)child);
  const ScratchArrays sc{smem, smem + N};
  build_child<M>(P, dm, 0, child, root, dst, sc, red, false, false, nullptr);
}

template <class M>
__device__ void expand_any(const PlanDesc &P, int l, unsigned long long child, float *smem,
                           float *red) {
  if (l == 0 && P.root_fused) expand_root_item<M>(P, child, smem, red);
  else expand_item<M>(P, l, child, smem, red);
}

// 256-thread CTAs (two per SM); a level that the host marks wide (long steps, at most one
// CTA per SM) takes kExpandWide threads per CTA, fewer particles per thread on its critical
// path.
#ifndef VOPP_EXPAND_WIDE
#define VOPP_EXPAND_WIDE 512
#endif
constexpr int kExpandWide = VOPP_EXPAND_WIDE;
template <int T>
__global__ void __launch_bounds__(T, (T <= 256) ? 2 : 1) k_expand(const PlanDesc *plans, StageTable st,
                                                              long long total) {
  extern __shared__ float smem[];
  __shared__ float red[kRedFloats];
  pdl_release_next();
  pdl_wait_prev();
  unsigned wg;
  if (copy_tail_block(st, wg)) return;
  for (long long item = blockIdx.x; item < total; item += wg) {
    const int pi = find_plan(st, item);
    const PlanDesc &P = plans[st.plan[pi]];
    const int l = st.levels ? st.levels[pi] : st.level;
    const unsigned long long child = (unsigned long long)(item - st.prefix[pi]);
    switch (P.kind) {
      case kNav: expand_any<NavModel>(P, l, child, smem, red); break;
      case kGrid: expand_any<GridModel>(P, l, child, smem, red); break;
      case kCrowd: expand_any<CrowdModel>(P, l, child, smem, red); break;
      default: expand_any<ToyModel>(P, l, child, smem, red); break;
    }
  }
}

// ---------------------------------------------------------------------------------------
// K2, vectorised: the expansion of the models whose particle is one or two words (NAV2D,
// GRID, TOY2), one kernel per model and vector width.  One warp builds one child: particle
// i of a child depends only on particle i of its parent (and on the branch observation),
// so a lane owns units of V consecutive particles (V = 4, 2 or 1: the largest that divides
// N, so that every node's store starts on a 16-, 8- or 4-byte boundary) from the parent
// load to the child store.  Pass 1 reads the parent's states and log weights as V-wide
// vectors, steps them, writes the child's states as V-wide streaming stores and parks the
// unnormalised base-2 log weights in the child's own log-weight store (the lane reads
// back only what it wrote), folding them into running max-shifted sums; the lanes merge
// their sums with shuffles (no barrier, no shared memory), and pass 2 rewrites the log
// weights normalised.  A CTA's warps take consecutive children, so siblings share their
// parent's lines in L2.
// ---------------------------------------------------------------------------------------
constexpr int kExpandVecThreads = VOPP_EXPAND_VEC_THREADS;
constexpr int kExpandVecWarps = kExpandVecThreads / 32;

template <int V> __device__ __forceinline__ void ldg_v(const float *p, float (&v)[V]) {
  if constexpr (V == 4) {
    const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else if constexpr (V == 2) {
    const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
    v[0] = t.x; v[1] = t.y;
  } else {
    v[0] = __ldg(p);
  }
}
template <int V> __device__ __forceinline__ void ldg_v(const int *p, int (&v)[V]) {
  if constexpr (V == 4) {
    const int4 t = __ldg(reinterpret_cast<const int4 *>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else if constexpr (V == 2) {
    const int2 t = __ldg(reinterpret_cast<const int2 *>(p));
    v[0] = t.x; v[1] = t.y;
  } else {
    v[0] = __ldg(p);
  }
}
// Child stores: plain write-back (1: streaming, evict-first; measured slower, 0.283 against
// 0.272 ms on the widest grid level).
#ifndef VOPP_EXPAND_STREAMING
#define VOPP_EXPAND_STREAMING 0
#endif
template <int V> __device__ __forceinline__ void st_child_v(float *p, const float (&v)[V]) {
  if constexpr (!VOPP_EXPAND_STREAMING) {
    if constexpr (V == 4) *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else if constexpr (V == 2) *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    else *p = v[0];
  } else if constexpr (V == 4) {
    __stcs(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
  } else if constexpr (V == 2) {
    __stcs(reinterpret_cast<float2 *>(p), make_float2(v[0], v[1]));
  } else {
    __stcs(p, v[0]);
  }
}
template <int V> __device__ __forceinline__ void st_child_v(int *p, const int (&v)[V]) {
  if constexpr (!VOPP_EXPAND_STREAMING) {
    if constexpr (V == 4) *reinterpret_cast<int4 *>(p) = make_int4(v[0], v[1], v[2], v[3]);
    else if constexpr (V == 2) *reinterpret_cast<int2 *>(p) = make_int2(v[0], v[1]);
    else *p = v[0];
  } else if constexpr (V == 4) {
    __stcs(reinterpret_cast<int4 *>(p), make_int4(v[0], v[1], v[2], v[3]));
  } else if constexpr (V == 2) {
    __stcs(reinterpret_cast<int2 *>(p), make_int2(v[0], v[1]));
  } else {
    __stcs(p, v[0]);
  }
}

// Step the V particles of unit u (particles u V .. u V + V - 1) of a NAV2D parent under
// branch (a, k): states in place, rewards r, base-2 log-likelihoods e.  Pairs of a unit share
// their Philox call; a single particle (V = 1) takes its half of its pair's words.
template <int V>
__device__ __forceinline__ void nav_unit(float (&x)[V], float (&y)[V], float (&r)[V], float (&e)[V],
                                         long long u, int a, uint32_t c1, unsigned long long kn,
                                         uint32_t key0, uint32_t key1, const NavModel::O &o,
                                         const DevModel &dm) {
  if constexpr (V >= 2) {
    const float dx = NavModel::dx_of(a), dy = NavModel::dy_of(a);
#pragma unroll
    for (int q = 0; q < V / 2; ++q) {
      const uint32_t p = (uint32_t)(u * (V / 2) + q);
      const uint4 w = philox(make_uint4(c1, p, (uint32_t)kn, (uint32_t)(kn >> 32)), key0, key1);
      float2 X = make_float2(x[2 * q], x[2 * q + 1]), Y = make_float2(y[2 * q], y[2 * q + 1]);
      bool t0, t1;
      const float2 rr = NavModel::step_pair(X, Y, dx, dy, w, t0, t1);
      const float2 ee = NavModel::loglik2_pair(X, Y, o);
      x[2 * q] = X.x; x[2 * q + 1] = X.y; y[2 * q] = Y.x; y[2 * q + 1] = Y.y;
      r[2 * q] = rr.x; r[2 * q + 1] = rr.y; e[2 * q] = ee.x; e[2 * q + 1] = ee.y;
    }
  } else {
    const uint32_t i = (uint32_t)u;
    const uint4 w = philox(make_uint4(c1, i >> 1, (uint32_t)kn, (uint32_t)(kn >> 32)), key0, key1);
    NavModel::S s{x[0], y[0]};
    r[0] = NavModel::step(s, a, (i & 1) ? w.z : w.x, (i & 1) ? w.w : w.y, dm);
    e[0] = NavModel::loglik2(s, a, o, dm);
    x[0] = s.x;
    y[0] = s.y;
  }
}

template <int V> __device__ __forceinline__ void st_v(float *p, const float (&v)[V]) {
  if constexpr (V == 4) *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
  else if constexpr (V == 2) *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
  else *p = v[0];
}
template <int V> __device__ __forceinline__ void ld_v(const float *p, float (&v)[V]) {
  if constexpr (V == 4) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else if constexpr (V == 2) {
    const float2 t = *reinterpret_cast<const float2 *>(p);
    v[0] = t.x; v[1] = t.y;
  } else {
    v[0] = *p;
  }
}

// A GRID child's action decided once (as the leaf's branch loops do): a sense action keeps
// the state, earns 0 and weighs by Z(o | s') from the model's log tables; a move changes
// one 4-bit field by one unless it is at its blocking value (east at x = 10 exits: x = 11
// and the terminal bit, +10); collect reads the cell's rock.  The same states, rewards and
// log-likelihoods as GridModel::step and GridModel::loglik2.
struct GridChild {
  int kind;                   // 0 sense, 1 move, 2 collect
  float e_null;               // log2 Z of a move's or collect's reading (0 if NULL, else -inf)
  int rk, rx, ry, want;       // sense: rock, its cell, the bit the reading agrees with
  bool valid;                 // sense: the reading is good or bad
  const float *lagree, *ldis; // sense: log2 Z when the reading agrees / disagrees, by d^2
  int shift, lo, span, delta, at_lim;
  float r_lim;
};
__device__ __forceinline__ GridChild grid_child(int a, GridModel::O o, const DevModel &dm) {
  GridChild g;
  g.e_null = (o.o == 0) ? 0.0f : -CUDART_INF_F;
  g.rk = g.rx = g.ry = g.want = 0;
  g.valid = false;
  g.lagree = g.ldis = nullptr;
  g.shift = g.lo = g.span = g.delta = g.at_lim = 0;
  g.r_lim = 0.0f;
  if (a >= 5) {
    g.kind = 0;
    g.rk = a - 5;
    g.rx = dm.rock_x[g.rk];
    g.ry = dm.rock_y[g.rk];
    g.valid = o.o == 1 || o.o == 2;
    g.want = (o.o == 1) ? 1 : 0;
    g.lagree = dm.lacc2;
    g.ldis = dm.l1macc2;   // = lacc2 + kGridD2
  } else if (a == 4) {
    g.kind = 2;
  } else {
    g.kind = 1;
    g.shift = (a < 2) ? 8 : 12;
    g.lo = (a == 0 || a == 2) ? 10 : 0;
    g.span = (a == 2) ? 5 : 0;
    g.delta = (a == 0) ? 0x100 : (a == 1) ? -0x100 : (a == 2) ? 0x1000 : -0x1000;
    g.at_lim = (a == 0) ? 0x10100 : 0;
    g.r_lim = (a == 0) ? 10.0f : 0.0f;
  }
  return g;
}
template <int V, int GK>
__device__ __forceinline__ void grid_child_unit(int (&sv)[V], float (&r)[V], float (&e)[V],
                                                const GridChild &g, const DevModel &dm) {
  if constexpr (GK == 0) {
    // log2 Z from [agree, disagree][d^2] (the model's log2 acc and log2(1 - acc) tables are
    // adjacent): disagree = the rock's bit differs from the one the reading agrees with
#pragma unroll
    for (int t = 0; t < V; ++t) {
      const int s = sv[t], dx = gx(s) - g.rx, dy = gy(s) - g.ry;
      const int miss = ((s >> g.rk) ^ g.want) & 1;
      const float lz = __ldg(g.lagree + (dx * dx + dy * dy + (miss << 8)));
      e[t] = g.valid ? lz : -CUDART_INF_F;
      r[t] = 0.0f;
    }
  } else if constexpr (GK == 1) {
#pragma unroll
    for (int t = 0; t < V; ++t) {
      const int s = sv[t];
      const bool term = gterm(s) != 0;
      const bool blk = (unsigned)(((s >> g.shift) & 0xF) - g.lo) <= (unsigned)g.span;
      sv[t] = term ? s : s + (blk ? g.at_lim : g.delta);
      r[t] = (term || !blk) ? 0.0f : g.r_lim;
      e[t] = g.e_null;
    }
  } else {
#pragma unroll
    for (int t = 0; t < V; ++t) {
      const int s = sv[t], x = gx(s);
      const int rk = (gterm(s) == 0 && x <= 10) ? __ldg(dm.rock_at + x + 11 * gy(s)) : -1;
      const bool good = rk >= 0 && ((s >> (rk & 7)) & 1);
      r[t] = (rk >= 0) ? (good ? 10.0f : -10.0f) : 0.0f;
      sv[t] = good ? (s & ~(1 << (rk & 7))) : s;
      e[t] = g.e_null;
    }
  }
}

// Unrolling of the two unit loops of a vectorised child (loads of several units in flight).
#ifndef VOPP_EXPAND_UNROLL1
#define VOPP_EXPAND_UNROLL1 1
#endif
#ifndef VOPP_EXPAND_UNROLL2
#define VOPP_EXPAND_UNROLL2 4
#endif
// Parent units a lane keeps in flight in pass 1 of a GRID / TOY2 child (4-particle units):
// config 3's level 3 took 275 us with plain loads, 230 / 224 / 234 us with 2 / 4 / 6.
#ifndef VOPP_K2_RING
#define VOPP_K2_RING 4
#endif
constexpr int kExpandUnroll1 = VOPP_EXPAND_UNROLL1, kExpandUnroll2 = VOPP_EXPAND_UNROLL2;
// Running sums of a child's pass 1 (per lane).
struct ChildPass {
  Kahan R, S1, S0, MX, MY;
  float m1, m0;
};

// Asynchronous 16-byte copies from global into shared memory (cp.async, through L2 only),
// committed and waited for by group; each lane reads back only what it copied itself.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K> __device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory");
}
// Per warp of a vectorised expansion: kRing slots × (states, log weights) × 32 lanes of one
// 4-particle unit each.  The loop's loads were its latency: with the next kRing - 1 units of
// a lane already on their way, no register holds them meanwhile.
constexpr int kRing = VOPP_K2_RING;
__shared__ __align__(16) uint4 s_ring[kExpandVecWarps][kRing][2][32];

// Pass 1 of a child over this lane's units (GK: the GRID action case, -1 for the generic
// step of the other models).
template <class M, int V, int GK>
__device__ __forceinline__ void child_pass1(const PlanDesc &P, const DevModel &dm, int l, int a,
                                            uint32_t c1, unsigned long long kn,
                                            const typename M::O o, const GridChild &gc,
                                            long long pb, long long cb, float *clw, ChildPass &cp) {
  const int lane = threadIdx.x & 31, units = P.N / V;
  // the mean particle is needed for the distance-softmax policy, a NAV2D policy only
  const bool want_mu = std::is_same<M, NavModel>::value && P.pi_mode == kPiNavDist;
  constexpr bool kNavM = std::is_same<M, NavModel>::value;
  const float *plw = P.plw[l] + pb;
  const float *sx = kNavM ? P.px[l] + pb : nullptr, *sy = kNavM ? P.py[l] + pb : nullptr;
  float *dx = kNavM ? P.px[l + 1] + cb : nullptr, *dy = kNavM ? P.py[l + 1] + cb : nullptr;
  const int *ss = kNavM ? nullptr : P.ps[l] + pb;
  int *ds = kNavM ? nullptr : P.ps[l + 1] + cb;
  // GRID / TOY2 with 4-particle units: the parent's states and log weights through the ring
  constexpr bool kRingOn = !kNavM && V == 4;
  if constexpr (kRingOn) {
#pragma unroll
    for (int k = 0; k < kRing - 1; ++k) {
      const int u = lane + 32 * k;
      if (u < units) {
        cp_async16(&s_ring[threadIdx.x >> 5][k][0][lane], ss + 4 * u);
        cp_async16(&s_ring[threadIdx.x >> 5][k][1][lane], plw + 4 * u);
      }
      cp_commit();   // (an empty group past the last unit keeps the count uniform)
    }
  }
#pragma unroll kExpandUnroll1
  for (int u = lane; u < units; u += 32) {
    const int i0 = u * V;
    float lw[V], r[V], e[V], X[V], Y[V];
    int sv[V];
    if constexpr (kRingOn) {
      // unit u is this lane's iteration it; the slot refilled now held iteration it - 1
      const int it = u >> 5, un = u + 32 * (kRing - 1), sn = (it + kRing - 1) % kRing;
      uint4 (*ring)[2][32] = s_ring[threadIdx.x >> 5];
      if (un < units) {
        cp_async16(&ring[sn][0][lane], ss + 4 * un);
        cp_async16(&ring[sn][1][lane], plw + 4 * un);
      }
      cp_commit();
      cp_wait<kRing - 1>();   // all but the newest kRing - 1 groups: unit u has landed
      const uint4 a4 = ring[it % kRing][0][lane], b4 = ring[it % kRing][1][lane];
      sv[0] = (int)a4.x; sv[1] = (int)a4.y; sv[2] = (int)a4.z; sv[3] = (int)a4.w;
      lw[0] = __uint_as_float(b4.x); lw[1] = __uint_as_float(b4.y);
      lw[2] = __uint_as_float(b4.z); lw[3] = __uint_as_float(b4.w);
    } else {
      ldg_v<V>(plw + i0, lw);
      if constexpr (kNavM) {
        ldg_v<V>(sx + i0, X);
        ldg_v<V>(sy + i0, Y);
      } else {
        ldg_v<V>(ss + i0, sv);
      }
    }
    if constexpr (kNavM) {
      nav_unit<V>(X, Y, r, e, u, a, c1, kn, P.key0, P.key1, o, dm);
      st_child_v<V>(dx + i0, X);
      st_child_v<V>(dy + i0, Y);
    } else {
      if constexpr (GK >= 0) {
        grid_child_unit<V, GK>(sv, r, e, gc, dm);
      } else {
#pragma unroll
        for (int t = 0; t < V; ++t) {
          typename M::S s{sv[t]};
          r[t] = M::step(s, a, 0u, 0u, dm);
          e[t] = M::loglik2(s, a, o, dm);
          sv[t] = s.s;
        }
      }
#pragma unroll
      for (int t = 0; t < V; ++t) X[t] = Y[t] = 0.f;
      st_child_v<V>(ds + i0, sv);
    }
    float L[V], rp = 0.f, cm1 = -CUDART_INF_F, cm0 = -CUDART_INF_F;
#pragma unroll
    for (int t = 0; t < V; ++t) {
      L[t] = fmaf(lw[t], kLog2e, e[t]);
      // a GRID sense step earns exactly 0: its reward sum is skipped
      if constexpr (GK != 0)
        if (lw[t] > -CUDART_INF_F) rp = fmaf(ex2(lw[t] * kLog2e), r[t], rp);
      cm1 = fmaxf(cm1, L[t]);
      cm0 = fmaxf(cm0, e[t]);
    }
    st_v<V>(clw + i0, L);            // parked until the normalisation pass
    // move the shifts to the unit's maxima, then add its shifted terms
    if (cm1 > cp.m1) {
      const float f = (cp.m1 > -CUDART_INF_F) ? ex2(cp.m1 - cm1) : 0.f;
      cp.S1.scale(f);
      if (want_mu) { cp.MX.scale(f); cp.MY.scale(f); }
      cp.m1 = cm1;
    }
    if (cm0 > cp.m0) {
      const float f = (cp.m0 > -CUDART_INF_F) ? ex2(cp.m0 - cm0) : 0.f;
      cp.S0.scale(f);
      cp.m0 = cm0;
    }
    float a1 = 0.f, a0 = 0.f, ax = 0.f, ay = 0.f;
    if (cp.m1 > -CUDART_INF_F) {
#pragma unroll
      for (int t = 0; t < V; ++t) {
        const float x1 = ex2(L[t] - cp.m1);   // L = -inf gives 0
        a1 += x1;
        if constexpr (std::is_same<M, NavModel>::value) {
          ax = fmaf(x1, X[t], ax);
          ay = fmaf(x1, Y[t], ay);
        }
      }
    }
    if (cp.m0 > -CUDART_INF_F) {
#pragma unroll
      for (int t = 0; t < V; ++t) a0 += ex2(e[t] - cp.m0);
    }
    cp.S1.add(a1); cp.S0.add(a0);
    if constexpr (GK != 0) cp.R.add(rp);
    if (want_mu) { cp.MX.add(ax); cp.MY.add(ay); }
  }
}

// One child of a vectorised expansion, by one warp (see above).
template <class M, int V>
__device__ __forceinline__ void expand_child_warp(const PlanDesc &P, const DevModel &dm, int l,
                                                  unsigned long long child) {
  const int lane = threadIdx.x & 31;
  const int N = P.N, AW = P.AW, W = P.W;
  unsigned long long parent;
  int slot;
  if (child < (1ull << 32)) {   // 32-bit division in the common case
    const uint32_t c32 = (uint32_t)child, p32 = c32 / (uint32_t)AW;
    parent = p32;
    slot = (int)(c32 - p32 * (uint32_t)AW);
  } else {
    parent = child / (unsigned long long)AW;
    slot = (int)(child - parent * (unsigned long long)AW);
  }
  const int a = slot / W, k = slot - (slot / W) * W;
  const unsigned long long kn = key_node(P, l, parent);
  const uint32_t c1 = key_level(P, l) | ((uint32_t)a << 8) | ((uint32_t)k << 16);
  const bool want_mu = P.pi_mode == kPiNavDist;
  const long long pb = (long long)parent * N, cb = (long long)child * N;
  float *clw = P.plw[l + 1] + cb;
  const int units = N / V;
  int j;
  const typename M::O o = branch_obs<M>(P, GNode<M>::at(P, l, (long long)parent), l, a, k, kn, dm, j);

  ChildPass cp;
  cp.R.init(); cp.S1.init(); cp.S0.init(); cp.MX.init(); cp.MY.init();
  cp.m1 = cp.m0 = -CUDART_INF_F;
  GridChild gc;
  if constexpr (std::is_same<M, GridModel>::value) {
    gc = grid_child(a, o, dm);
    if (gc.kind == 0) child_pass1<M, V, 0>(P, dm, l, a, c1, kn, o, gc, pb, cb, clw, cp);
    else if (gc.kind == 1) child_pass1<M, V, 1>(P, dm, l, a, c1, kn, o, gc, pb, cb, clw, cp);
    else child_pass1<M, V, 2>(P, dm, l, a, c1, kn, o, gc, pb, cb, clw, cp);
  } else {
    child_pass1<M, V, -1>(P, dm, l, a, c1, kn, o, gc, pb, cb, clw, cp);
  }
  // the lanes' sums at the warp's largest shifts
  float w1 = cp.m1, w0 = cp.m0, s1 = cp.S1.value(), mx = cp.MX.value(), my = cp.MY.value();
  float s0 = cp.S0.value();
  warp_lse2(w1, s1, mx);
  float dummy = 0.f;
  warp_lse2(w0, s0, dummy);
  my *= (cp.m1 > -CUDART_INF_F) ? ex2(cp.m1 - w1) : 0.f;
  my = warp_sum(my);
  const float rbar = warp_sum(cp.R.value());
  const float lse2 = (s1 > 0.f) ? w1 + lg2(s1) : -CUDART_INF_F;   // base 2
  if (lse2 > -CUDART_INF_F) {
    const float off = -kLn2 * lse2;   // natural log weight = ln 2 (L - lse2)
#pragma unroll kExpandUnroll2
    for (int u = lane; u < units; u += 32) {
      const int i0 = u * V;
      float L[V];
      ld_v<V>(clw + i0, L);
#pragma unroll
      for (int t = 0; t < V; ++t) L[t] = fmaf(L[t], kLn2, off);
      st_child_v<V>(clw + i0, L);
    }
  } else {   // no weight left: every child particle has log weight -inf
    float L[V];
#pragma unroll
    for (int t = 0; t < V; ++t) L[t] = -CUDART_INF_F;
    for (int u = lane; u < units; u += 32) st_child_v<V>(clw + u * V, L);
  }
  if (lane == 0) {
    float lom;
    if (P.branch_mode == kEnumerate) lom = kLn2 * lse2;
    else lom = (lse2 > -CUDART_INF_F) ? __logf((float)N) + kLn2 * (lse2 - (w0 + lg2(s0))) : -CUDART_INF_F;
    const int cl = l + 1;
    if (cl <= P.D - 2) P.cnt[cl][child] = 0u;   // completion counter of the new node
    P.rbar[cl][child] = rbar;
    P.lom[cl][child] = lom;
    if (want_mu && P.mu[cl]) {
      float2 mu = make_float2(0.f, 0.f);
      if (s1 > 0.f) mu = make_float2(mx / s1, my / s1);
      P.mu[cl][2 * child] = mu.x;
      P.mu[cl][2 * child + 1] = mu.y;
    }
    if (P.rep[cl]) P.rep[cl][child] = j;
    if (P.obs[cl]) {
      const float2 of = M::obs_f2(o);
      P.obs[cl][2 * child] = of.x;
      P.obs[cl][2 * child + 1] = of.y;
    }
  }
}

// Per model: the resident CTAs per SM the register budget is set for (128-thread CTAs).
#ifndef VOPP_EXPAND_NAV_MINBLOCKS
#define VOPP_EXPAND_NAV_MINBLOCKS 6
#endif
#ifndef VOPP_EXPAND_GRID_MINBLOCKS
#define VOPP_EXPAND_GRID_MINBLOCKS 8
#endif
template <int K> struct ExpandModel;
template <> struct ExpandModel<kNav> { using type = NavModel; static constexpr int kMinBlocks = VOPP_EXPAND_NAV_MINBLOCKS; };
template <> struct ExpandModel<kGrid> { using type = GridModel; static constexpr int kMinBlocks = VOPP_EXPAND_GRID_MINBLOCKS; };
template <> struct ExpandModel<kToy> { using type = ToyModel; static constexpr int kMinBlocks = VOPP_EXPAND_GRID_MINBLOCKS; };

// Work items: the children of every plan of the stage at level l + 1, one per warp.
template <int K, int V>
__global__ void __launch_bounds__(kExpandVecThreads, ExpandModel<K>::kMinBlocks)
k_expand_vec(const PlanDesc *plans, StageTable st, long long total) {
  using M = typename ExpandModel<K>::type;
  pdl_release_next();
  pdl_wait_prev();
  unsigned wg;
  if (copy_tail_block(st, wg)) return;
  const long long wid = threadIdx.x >> 5;
  for (long long item = (long long)blockIdx.x * kExpandVecWarps + wid; item < total;
       item += (long long)wg * kExpandVecWarps) {
    const int pi = find_plan(st, item);
    const PlanDesc &P = plans[st.plan[pi]];
    const int l = st.levels ? st.levels[pi] : st.level;
    expand_child_warp<M, V>(P, *P.model, l, (unsigned long long)(item - st.prefix[pi]));
  }
}

// ---------------------------------------------------------------------------------------
// K3: leaf expansion of one level-(D-1) node, fused with its backup.
// ---------------------------------------------------------------------------------------
// Compile-time tuning of the leaf loop (results do not depend on them beyond the rounding
// order of the compensated sums):
//   VOPP_LEAF_CHUNK      pairs per lane between two compensated adds of the generic loops
//                        (TOY2; the log-domain path's rescales)
//   VOPP_LEAF_CHUNK_LIN  pairs per lane between two compensated adds, NAV2D linear sums
//   VOPP_GRID_CHUNK      the same for the GRID branch loops (sense, move, collect)
//   VOPP_SELF_CHUNK      particles per lane between two compensated adds, CROWD
//   VOPP_LOG_COLD_NAV / VOPP_LOG_COLD_GRID  1: the log-domain fallback is an out-of-line call
//   VOPP_LEAF_NAV_MAXREG registers per thread of the NAV2D leaf kernel (72: seven 128-thread
//                        CTAs per SM); VOPP_LEAF_GRID_MAXREG: GRID (72: its shared memory
//                        allows seven CTAs per SM, which 72 registers still fit; 64 spilled,
//                        4.28 against 4.19 ms on the depth-4 grid plan); VOPP_LEAF_TOY_MAXREG: TOY2 (64);
//                        VOPP_LEAF_CROWD_MINBLOCKS: resident 160-thread CROWD CTAs per SM (3)
#ifndef VOPP_LEAF_CHUNK
#define VOPP_LEAF_CHUNK 4
#endif
#ifndef VOPP_LEAF_NAV_MAXREG
#define VOPP_LEAF_NAV_MAXREG 72
#endif
#ifndef VOPP_LEAF_GRID_MAXREG
#define VOPP_LEAF_GRID_MAXREG 72
#endif
#ifndef VOPP_LEAF_TOY_MAXREG
#define VOPP_LEAF_TOY_MAXREG 64
#endif
#ifndef VOPP_LEAF_CROWD_MINBLOCKS
#define VOPP_LEAF_CROWD_MINBLOCKS 3
#endif
constexpr int kLeafChunk = VOPP_LEAF_CHUNK;
#ifndef VOPP_LEAF_CHUNK_LIN
#define VOPP_LEAF_CHUNK_LIN 4
#endif
constexpr int kLeafChunkLin = VOPP_LEAF_CHUNK_LIN;   // pairs per compensated add, linear sums
#ifndef VOPP_SELF_CHUNK
#define VOPP_SELF_CHUNK 1
#endif
constexpr int kSelfChunk = VOPP_SELF_CHUNK;          // particles per compensated add, CROWD
#ifndef VOPP_GRID_CHUNK
#define VOPP_GRID_CHUNK 4
#endif
constexpr int kGridChunk = VOPP_GRID_CHUNK;          // pairs per compensated add, GRID loops
#ifndef VOPP_LOG_COLD_GRID
#define VOPP_LOG_COLD_GRID 1
#endif
#ifndef VOPP_LOG_COLD_NAV
#define VOPP_LOG_COLD_NAV 1
#endif
template <class M> struct kLogCold { static constexpr bool value = false; };
template <> struct kLogCold<GridModel> { static constexpr bool value = VOPP_LOG_COLD_GRID != 0; };
template <> struct kLogCold<NavModel> { static constexpr bool value = VOPP_LOG_COLD_NAV != 0; };
constexpr int kLeafChunkLog = 1;                     // pairs per rescale, log-domain sums

// Running max-shifted sums in base 2: S = sum 2^(L - m) and H = sum 2^(L - m) h, compensated.
struct ShiftedSum {
  float m;
  Kahan S, H;
  __device__ __forceinline__ void init() { m = -CUDART_INF_F; S.init(); H.init(); }
  // Move the shift to max(m, cm); returns the new shift.
  __device__ __forceinline__ float shift_to(float cm) {
    const float nm = fmaxf(m, cm);
    if (nm > m) {
      const float f = (m > -CUDART_INF_F) ? ex2(m - nm) : 0.f;
      S.scale(f);
      H.scale(f);
      m = nm;
    }
    return m;
  }
};

// One leaf branch (slot a*W + k of a level-(D-1) node) by one warp.  The node's particles
// are in shared memory with base-2 log weights; every lane steps Philox pairs p = lane,
// lane + 32, ... and keeps running sums over L = lw + log2 Z (child weights, heuristic) and
// over log2 Z (the proposal normaliser of omega), rescaled once per chunk of pairs.
// GRID: the leaf heuristic per column x (it depends on x alone), filled by each leaf CTA
// with the same arithmetic as GridModel::heuristic.
// GRID leaf tables by cell c = x + 16 y (x <= 11, y <= 10, so c < 172): Z of a sense of each
// rock (agreeing, disagreeing reading) at the cell's squared distance to it, heuristic (0 at
// the exited column x = 11) and the rock on the cell (-1 if none).  Small enough, with the
// 16-byte node pairs, for seven 128-thread leaf CTAs per SM.
constexpr int kGridCells = 172;
__shared__ float2 s_grid_zc[8 * kGridCells];
__shared__ float s_grid_hc[kGridCells];
__shared__ signed char s_grid_rockc[kGridCells];
// (s >> 8) & 0xFF as one byte permute (byte 1 of s, zero bytes above it) instead of a shift
// and a mask: depth-4 grid leaf 4.91 -> 4.60 ms
__device__ __forceinline__ int gcell(int s) { return (int)__byte_perm((unsigned)s, 0u, 0x4441u); }

// The leaf heuristic (GRID: from the CTA's column table).
template <class M>
__device__ __forceinline__ float leaf_heuristic(const typename M::S &s, float log2g, float a0,
                                                float b0, bool hz) {
  if constexpr (std::is_same<M, GridModel>::value) return s_grid_hc[gcell(s.s)];
  else return M::heuristic(s, log2g, a0, b0, hz);
}

// Leaf sums of one branch, log domain: S1 = sum 2^(L - m1) with L = lw2 + log2 Z and a
// running shift m1, S0 = sum 2^(log2 Z - m0) with its own shift, H = sum 2^(L - m1) h, and
// the reward mean.  Exact in relative terms however small the weights: the path for
// enumerated observations, and for the rare branch whose linear sums are too small.
template <class M>
__device__ __forceinline__ void leaf_sums_log(const PlanDesc &P, const DevModel &dm,
                                           const SNode<M> &nb, int a, uint32_t c1,
                                           unsigned long long kn, const typename M::O o,
                                           float &rbar_out, float &lom_out, float &v_out) {
  const int lane = threadIdx.x & 31, N = P.N;
  const float log2g = P.log2_gamma, h_a0 = P.h_a0, h_b0 = P.h_b0;
  const bool hz = P.h_zero != 0;
  const uint32_t key0 = P.key0, key1 = P.key1;
  const uint32_t c2 = (uint32_t)kn, c3 = (uint32_t)(kn >> 32);
  ShiftedSum A1, A0;
  A1.init();
  A0.init();
  Kahan R;
  R.init();
  const int npairs = (N + 1) >> 1;
  if constexpr (M::kPairPacked) {
    // both particles of a pair through one two-wide instruction stream
    const float dx = NavModel::dx_of(a), dy = NavModel::dy_of(a);
    for (int base = lane; base < npairs; base += 32 * kLeafChunkLog) {
      float2 L[kLeafChunkLog], E[kLeafChunkLog], Hh[kLeafChunkLog];
      float2 rsum = make_float2(0.f, 0.f);
      float cm1 = -CUDART_INF_F, cm0 = -CUDART_INF_F;
#pragma unroll
      for (int c = 0; c < kLeafChunkLog; ++c) {
        const int p = base + 32 * c;
        L[c] = E[c] = bc2(-CUDART_INF_F);
        Hh[c] = bc2(0.f);
        if (p < npairs) {
          const uint4 w = philox(make_uint4(c1, (uint32_t)p, c2, c3), key0, key1);
          const float4 xy = nb.xy(p);              // (x0, x1, y0, y1)
          const float4 b = nb.B[p];                // (lw2_0, lw2_1, w_0, w_1)
          float2 X = make_float2(xy.x, xy.y), Y = make_float2(xy.z, xy.w);
          bool t0, t1;
          const float2 r = NavModel::step_pair(X, Y, dx, dy, w, t0, t1);
          const float2 e = NavModel::loglik2_pair(X, Y, o_nav(o));
          const bool v1 = 2 * p + 1 < N;
          L[c] = add2(make_float2(b.x, b.y), e);   // the odd-N pad slot has lw2 = -inf
          E[c] = make_float2(e.x, v1 ? e.y : -CUDART_INF_F);
          Hh[c] = NavModel::heuristic_pair(X, Y, t0, t1, log2g, h_a0, h_b0, hz);
          rsum = fma2(make_float2(b.z, b.w), r, rsum);   // pad slot: w = 0
          cm1 = fmax3(cm1, L[c].x, L[c].y);
          cm0 = fmax3(cm0, E[c].x, E[c].y);
        }
      }
      const float m1 = A1.shift_to(cm1), m0 = A0.shift_to(cm0);
      float2 s1 = bc2(0.f), h1 = bc2(0.f), s0 = bc2(0.f);
      if (m1 > -CUDART_INF_F) {
#pragma unroll
        for (int c = 0; c < kLeafChunkLog; ++c) {
          const float2 d = add2(L[c], bc2(-m1));
          const float2 x1 = make_float2(ex2(d.x), ex2(d.y));   // L = -inf gives 0
          s1 = add2(s1, x1);
          h1 = fma2(x1, Hh[c], h1);
        }
      }
      if (m0 > -CUDART_INF_F) {
#pragma unroll
        for (int c = 0; c < kLeafChunkLog; ++c) {
          const float2 d = add2(E[c], bc2(-m0));
          s0 = add2(s0, make_float2(ex2(d.x), ex2(d.y)));
        }
      }
      A1.S.add(s1.x + s1.y);
      A1.H.add(h1.x + h1.y);
      A0.S.add(s0.x + s0.y);
      R.add(rsum.x + rsum.y);
    }
  } else {
  // a self-drawing model's step is long: one pair per chunk keeps the unrolled loop small
  // enough for the instruction cache
  constexpr int kCh = 1;
  for (int base = lane; base < npairs; base += 32 * kCh) {
    float L[2 * kCh], E[2 * kCh], Hh[2 * kCh];
    float cm1 = -CUDART_INF_F, cm0 = -CUDART_INF_F, rsum = 0.f;
#pragma unroll
    for (int c = 0; c < kCh; ++c) {
      const int p = base + 32 * c;
      L[2 * c] = L[2 * c + 1] = E[2 * c] = E[2 * c + 1] = -CUDART_INF_F;
      Hh[2 * c] = Hh[2 * c + 1] = 0.f;
      if (p < npairs) {
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        if (M::kStochastic) {   // purpose 0 (transition): counter word 0 is the pair index
          w = philox(make_uint4(c1, (uint32_t)p, c2, c3), key0, key1);
        }
        typename M::S s0, s1;
        nb.get_pair(p, s0, s1);
        const float4 b = nb.pairB(p);      // (lw2_0, lw2_1, w_0, w_1)
        const DrawCtx dc{P.key0, P.key1, kPurposeTransition, c1, kn};
        const float r0 = step_particle<M>(s0, a, w, 2 * p, dc, dm);
        const float r1 = step_particle<M>(s1, a, w, 2 * p + 1, dc, dm);
        const float e0 = M::loglik2(s0, a, o, dm), e1 = M::loglik2(s1, a, o, dm);
        const bool v1 = 2 * p + 1 < N;
        L[2 * c] = b.x + e0;
        E[2 * c] = e0;
        Hh[2 * c] = leaf_heuristic<M>(s0, log2g, h_a0, h_b0, hz);
        L[2 * c + 1] = b.y + e1;           // the odd-N pad slot has lw2 = -inf
        E[2 * c + 1] = v1 ? e1 : -CUDART_INF_F;
        Hh[2 * c + 1] = leaf_heuristic<M>(s1, log2g, h_a0, h_b0, hz);
        rsum = fmaf(b.z, r0, rsum);
        rsum = fmaf(b.w, r1, rsum);        // pad slot: w = 0
        cm1 = fmaxf(cm1, fmaxf(L[2 * c], L[2 * c + 1]));
        cm0 = fmaxf(cm0, fmaxf(E[2 * c], E[2 * c + 1]));
      }
    }
    const float m1 = A1.shift_to(cm1), m0 = A0.shift_to(cm0);
    float s1 = 0.f, h1 = 0.f, s0 = 0.f;
    if (m1 > -CUDART_INF_F) {
#pragma unroll
      for (int t = 0; t < 2 * kCh; ++t) {
        const float x1 = ex2(L[t] - m1);    // L = -inf gives 0
        s1 += x1;
        h1 = fmaf(x1, Hh[t], h1);
      }
    }
    if (m0 > -CUDART_INF_F) {
#pragma unroll
      for (int t = 0; t < 2 * kCh; ++t) s0 += ex2(E[t] - m0);
    }
    A1.S.add(s1);
    A1.H.add(h1);
    A0.S.add(s0);
    R.add(rsum);
  }
  }
  float m1 = A1.m, s1 = A1.S.value(), h1 = A1.H.value();
  float m0 = A0.m, s0 = A0.S.value(), h0 = 0.f;
  warp_lse2(m1, s1, h1);
  warp_lse2(m0, s0, h0);
  const float rbar = warp_sum(R.value());
  const float lse1 = (s1 > 0.f) ? kLn2 * (m1 + lg2(s1)) : -CUDART_INF_F;
  if (P.branch_mode == kEnumerate) lom_out = lse1;
  else lom_out = (lse1 > -CUDART_INF_F) ? __logf((float)N) + lse1 - kLn2 * (m0 + lg2(s0)) : -CUDART_INF_F;
  v_out = (s1 > 0.f) ? h1 / s1 : 0.f;
  rbar_out = rbar;
}

// GRID leaf branches, with the action's case decided once per branch.  A sense action
// keeps every state and earns 0, so only Z (from the shared-memory table by d^2 and
// agreement) and h are per particle; a move changes one 4-bit field of the packed state by
// one unless the field is at its blocking range [lo, lo + span] (east at x = 10 exits
// instead: x = 11 and the terminal bit, +10); collect keeps the cell and reads its rock.  The
// same states and rewards as GridModel::step, which the other kernels use.  A move's or
// collect's reading is NULL (Z = 1) and a sense reading good or bad; any other reading has
// Z = 0 everywhere and is left to the log-domain path (false returned).
// sense of rock rk: mask = the rock's bit, fm = mask when the reading is "good" (so that
// (s ^ fm) & mask is nonzero exactly when the reading disagrees with the rock's bit: one
// three-input logic op)
struct GridSense { int mask, fm; const float2 *zc; };
// move: the moved field in place and the terminal bit (fmask), the blocking range's start
// and span shifted to the field; a terminal state's masked value lies above every range, so
// it is never blocked
struct GridMove { int fmask, lo_s, span_s, delta, at_lim; float r_lim; };
struct GridSums { float s0, s1, h1, rs; };


__device__ __forceinline__ void grid_sense_one(int sv, float w, const GridSense &g, GridSums &t) {
  const int c = gcell(sv);
  const bool miss = ((sv ^ g.fm) & g.mask) != 0;
  const float2 zz = g.zc[c];
  const float z = miss ? zz.y : zz.x;
  const float wz = w * z;
  t.s0 += z;
  t.s1 += wz;
  t.h1 = fmaf(wz, s_grid_hc[c], t.h1);
}
__device__ __forceinline__ void grid_move_one(int sv, float w, const GridMove &g, GridSums &t) {
  const bool term = gterm(sv) != 0;
  const bool blk = (unsigned)((sv & g.fmask) - g.lo_s) <= (unsigned)g.span_s;
  const int ns = term ? sv : sv + (blk ? g.at_lim : g.delta);
  const float r = blk ? g.r_lim : 0.0f;
  t.s0 += 1.0f;
  t.s1 += w;
  t.h1 = fmaf(w, s_grid_hc[gcell(ns)], t.h1);
  t.rs = fmaf(w, r, t.rs);
}
__device__ __forceinline__ void grid_collect_one(int sv, float w, GridSums &t) {
  const int c = gcell(sv);
  const int rk = gterm(sv) ? -1 : s_grid_rockc[c];
  const float h = s_grid_hc[c];
  const bool good = rk >= 0 && ((sv >> (rk & 7)) & 1);
  const float r = (rk >= 0) ? (good ? 10.0f : -10.0f) : 0.0f;
  t.s0 += 1.0f;
  t.s1 += w;
  t.h1 = fmaf(w, h, t.h1);
  t.rs = fmaf(w, r, t.rs);
}

// Two independent Kahan sums in the lanes of a float2 (the subtractions as exact FMAs by -1).
struct Kahan2 {
  float2 s, c;
  __device__ __forceinline__ void init() { s = c = bc2(0.f); }
  __device__ __forceinline__ void add(float2 v) {
    const float2 y = fma2(c, bc2(-1.f), v);
    const float2 t = add2(s, y);
    c = fma2(y, bc2(-1.f), fma2(s, bc2(-1.f), t));
    s = t;
  }
};

// Every whole pair through `one`: when the pairs make whole chunks of kGridChunk pairs per
// lane, a chunk between compensated adds with no bounds test; otherwise one pair per
// compensated add; then the last particle of an odd N (no pad particle is stepped).  kR: a move or
// collect branch -- its reading is NULL, so Z = 1 for every particle and S0 = N exactly (not
// summed), and its rewards are summed; a sense branch earns nothing.  The compensated sums
// run two at a time: (S0, S1) for sense, (S1, H) for move and collect.
template <bool kR, class F>
__device__ __forceinline__ void grid_pairs(const SNode<GridModel> &nb, int N, F one, Kahan &S0,
                                           Kahan &S1, Kahan &H, Kahan &R) {
  const int lane = threadIdx.x & 31, nfull = N >> 1;
  constexpr int kCh = kGridChunk;
  Kahan2 K;
  K.init();
  auto fold = [&](const GridSums &t) {
    if (kR) {
      K.add(make_float2(t.s1, t.h1));
      R.add(t.rs);
    } else {
      K.add(make_float2(t.s0, t.s1));
      H.add(t.h1);
    }
  };
  if (nfull % (32 * kCh) == 0) {   // whole chunks only
    for (int base = lane; base < nfull; base += 32 * kCh) {
      GridSums t{0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int c = 0; c < kCh; ++c) {
        const int p = base + 32 * c;
        const int2 st = nb.A[p];
        const float2 b = nb.W2[p];                 // (w_0, w_1)
        one(st.x, b.x, t);
        one(st.y, b.y, t);
      }
      fold(t);
    }
  } else {   // a pair at a time
    for (int p = lane; p < nfull; p += 32) {
      GridSums t{0.f, 0.f, 0.f, 0.f};
      const int2 st = nb.A[p];
      const float2 b = nb.W2[p];
      one(st.x, b.x, t);
      one(st.y, b.y, t);
      fold(t);
    }
  }
  if ((N & 1) && lane == 0) {
    GridSums t{0.f, 0.f, 0.f, 0.f};
    one(nb.A[nfull].x, nb.W2[nfull].x, t);
    fold(t);
  }
  if (kR) {
    S0.s = (lane == 0) ? (float)N : 0.f;   // the lanes' shares of S0 = N
    S0.c = 0.f;
    S1.s = K.s.x; S1.c = K.c.x;
    H.s = K.s.y; H.c = K.c.y;
  } else {
    S0.s = K.s.x; S0.c = K.c.x;
    S1.s = K.s.y; S1.c = K.c.y;
  }
}

__device__ __forceinline__ bool grid_branch_sums(const PlanDesc &P, const DevModel &dm,
                                                 const SNode<GridModel> &nb, int a,
                                                 GridModel::O o, Kahan &S0, Kahan &S1,
                                                 Kahan &H, Kahan &R) {
  const int N = P.N;
  if (a >= 5) {
    if (o.o != 1 && o.o != 2) return false;
    const int rk = a - 5;
    const GridSense g{1 << rk, (o.o == 1) ? (1 << rk) : 0, s_grid_zc + rk * kGridCells};
    grid_pairs<false>(nb, N, [&](int sv, float w, GridSums &t) { grid_sense_one(sv, w, g, t); },
                      S0, S1, H, R);    // R stays 0: a sense action earns nothing
    return true;
  }
  if (o.o != 0) return false;
  if (a == 4) {
    grid_pairs<true>(nb, N, [&](int sv, float w, GridSums &t) { grid_collect_one(sv, w, t); },
                     S0, S1, H, R);
    return true;
  }
  // a = 0 E, 1 W, 2 N, 3 S; N is blocked at y >= 10
  const int sh = (a < 2) ? 8 : 12;
  const GridMove g{(0xF << sh) | 0x10000, ((a == 0 || a == 2) ? 10 : 0) << sh, ((a == 2) ? 5 : 0) << sh,
                   (a == 0) ? 0x100 : (a == 1) ? -0x100 : (a == 2) ? 0x1000 : -0x1000,
                   (a == 0) ? 0x10100 : 0, (a == 0) ? 10.0f : 0.0f};
  grid_pairs<true>(nb, N, [&](int sv, float w, GridSums &t) { grid_move_one(sv, w, g, t); },
                   S0, S1, H, R);
  return true;
}

// The log-domain sums out of line, for kernels whose hot loop should keep the instruction
// cache to itself.
template <class M>
__device__ __noinline__ void leaf_sums_log_cold(const PlanDesc &P, const DevModel &dm,
                                                const SNode<M> &nb, int a, uint32_t c1,
                                                unsigned long long kn, const typename M::O o,
                                                float &rbar_out, float &lom_out, float &v_out) {
  leaf_sums_log<M>(P, dm, nb, a, c1, kn, o, rbar_out, lom_out, v_out);
}

// Round keys of the plan whose node a leaf CTA holds (filled once per node): the NAV2D branch
// loop reads them instead of adding the key increments in every Philox call (296 against
// 299 us, 102.7 against 107.3 issued per particle-step).
__shared__ uint2 s_leaf_rk[10];

// Linear sums of sampled-observation branches: z_i = Z(o | s'_i) up to a factor common to
// the branch (the model's zlin), S0 = sum z_i, S1 = sum w_i z_i, H = sum w_i z_i h_i, so
// that omega = N S1 / S0 and V = H / S1 need neither a logarithm per particle nor a running
// maximum.  The weights w_i are the node's normalised linear weights.  A particle whose z_i
// or w_i z_i flushes to zero loses at most 2^-126 x 288.5 (the largest z) of a sum, N x that
// over the branch, far below 2^-64: when S1 is at least 2^-64 the sums are exact to FP32
// rounding; otherwise (false returned, the same in every lane) the caller recomputes the
// branch in the log domain.
constexpr float kLinMinS1 = 5.42101086e-20f;   // 2^-64
// The NAV2D branch loop of leaf_sums_lin: every lane steps Philox pairs p = lane, lane + 32,
// ... (kLeafChunkLin pairs per compensated add) from the node's scaled positions and live
// masks; kFull: N is a multiple of 64 kLeafChunkLin, so every chunk is whole and there is no
// pad slot (N = 1024: 296 -> 281 us on its own).  With the masks and scaled positions the
// terminal state, the reward and the heuristic's zeroing are FMA operands instead of
// compares and selects (with the hardware square root, 296 -> 259 us).
template <bool kFull>
__device__ __forceinline__ void nav_lin_loop(const SNode<NavModel> &nb, int N, int a,
                                             uint32_t c1, uint32_t c2, uint32_t c3,
                                             NavModel::O o, float log2g, float h_a0, float h_b0,
                                             bool hz, Kahan &S0, Kahan &S1, Kahan &H, Kahan &R) {
  const int lane = threadIdx.x & 31, npairs = (N + 1) >> 1;
  const float dx16 = 0.0625f * NavModel::dx_of(a), dy16 = 0.0625f * NavModel::dy_of(a);
  const float a0 = hz ? 0.0f : h_a0, b0 = hz ? 0.0f : h_b0;   // forced-zero heuristic: h = 0
  for (int base = lane; base < npairs; base += 32 * kLeafChunkLin) {
    float2 s0 = bc2(0.f), s1 = bc2(0.f), h1 = bc2(0.f), rs = bc2(0.f);
#pragma unroll
    for (int c = 0; c < kLeafChunkLin; ++c) {
      const int p = base + 32 * c;
      if (kFull || p < npairs) {
        const uint4 w = philox_rk(make_uint4(c1, (uint32_t)p, c2, c3), s_leaf_rk);
        const float4 xy = nb.A16(p);             // (x0, x1, y0, y1) / 16
        const float4 b = nb.B[p];                // (lw2_0, lw2_1, w_0, w_1)
        const float2 m = nb.Mk[p];
        float2 X = make_float2(xy.x, xy.y), Y = make_float2(xy.z, xy.w), gm;
        const float2 r = NavModel::step_pair16(X, Y, dx16, dy16, w, m, gm);
        float2 z = NavModel::zlin_pair16(X, Y, o);
        if (!kFull) z.y = (2 * p + 1 < N) ? z.y : 0.f;       // the odd-N pad slot
        const float2 wt = make_float2(b.z, b.w); // pad slot: w = 0
        const float2 hh = NavModel::heuristic_pair16(X, Y, gm, log2g, a0, b0);
        const float2 wz = mul2(wt, z);
        s0 = add2(s0, z);
        s1 = add2(s1, wz);
        h1 = fma2(wz, hh, h1);
        rs = fma2(wt, r, rs);
      }
    }
    S0.add(s0.x + s0.y);
    S1.add(s1.x + s1.y);
    H.add(h1.x + h1.y);
    R.add(rs.x + rs.y);
  }
}

template <class M>
__device__ __forceinline__ bool leaf_sums_lin(const PlanDesc &P, const DevModel &dm,
                                              const SNode<M> &nb, int a, uint32_t c1,
                                              unsigned long long kn, const typename M::O o,
                                              float &rbar_out, float &lom_out, float &v_out) {
  const int lane = threadIdx.x & 31, N = P.N;
  const float log2g = P.log2_gamma, h_a0 = P.h_a0, h_b0 = P.h_b0;
  const bool hz = P.h_zero != 0;
  const uint32_t key0 = P.key0, key1 = P.key1;
  const uint32_t c2 = (uint32_t)kn, c3 = (uint32_t)(kn >> 32);
  Kahan S0, S1, H, R;
  S0.init();
  S1.init();
  H.init();
  R.init();
  const int npairs = (N + 1) >> 1;
  if constexpr (M::kPairPacked) {
    // whole chunks (N a multiple of 64 kLeafChunkLin): no bounds test and no pad slot
    if ((N % (64 * kLeafChunkLin)) == 0)
      nav_lin_loop<true>(nb, N, a, c1, c2, c3, o_nav(o), log2g, h_a0, h_b0, hz, S0, S1, H, R);
    else
      nav_lin_loop<false>(nb, N, a, c1, c2, c3, o_nav(o), log2g, h_a0, h_b0, hz, S0, S1, H, R);
  } else if constexpr (std::is_same<M, GridModel>::value) {
    if (!grid_branch_sums(P, dm, nb, a, o, S0, S1, H, R)) return false;
  } else if (SelfDraw<M>::value) {
    // a self-drawing step is long and needs no pair words: one particle per loop body (the
    // instruction cache), kSelfChunk particles per lane between compensated adds
    const DrawCtx dc{key0, key1, kPurposeTransition, c1, kn};
    for (int base = lane; base < N; base += 32 * kSelfChunk) {
      float s0 = 0.f, s1 = 0.f, h1 = 0.f, rs = 0.f;
#pragma unroll 1
      for (int c = 0; c < kSelfChunk; ++c) {
        const int i = base + 32 * c;
        if (i < N) {
          typename M::S x = nb.get(i);
          const float wi = nb.w(i);
          const float r = step_particle<M>(x, a, make_uint4(0u, 0u, 0u, 0u), i, dc, dm);
          const float z = M::zlin(x, a, o, dm);
          const float wz = wi * z;
          s0 += z;
          s1 += wz;
          h1 = fmaf(wz, leaf_heuristic<M>(x, log2g, h_a0, h_b0, hz), h1);
          rs = fmaf(wi, r, rs);
        }
      }
      S0.add(s0);
      S1.add(s1);
      H.add(h1);
      R.add(rs);
    }
  } else {
    constexpr int kCh = SelfDraw<M>::value ? 1 : kLeafChunk;
    for (int base = lane; base < npairs; base += 32 * kCh) {
      float s0 = 0.f, s1 = 0.f, h1 = 0.f, rs = 0.f;
#pragma unroll
      for (int c = 0; c < kCh; ++c) {
        const int p = base + 32 * c;
        if (p < npairs) {
          uint4 w = make_uint4(0u, 0u, 0u, 0u);
          if (M::kStochastic) w = philox(make_uint4(c1, (uint32_t)p, c2, c3), key0, key1);
          typename M::S x0, x1;
          nb.get_pair(p, x0, x1);
          const float4 b = nb.pairB(p);      // (lw2_0, lw2_1, w_0, w_1)
          const DrawCtx dc{key0, key1, kPurposeTransition, c1, kn};
          const float r0 = step_particle<M>(x0, a, w, 2 * p, dc, dm);
          const float r1 = step_particle<M>(x1, a, w, 2 * p + 1, dc, dm);
          const float z0 = M::zlin(x0, a, o, dm);
          const float z1 = (2 * p + 1 < N) ? M::zlin(x1, a, o, dm) : 0.f;
          const float wz0 = b.z * z0, wz1 = b.w * z1;   // pad slot: w = 0
          s0 += z0 + z1;
          s1 += wz0 + wz1;
          h1 = fmaf(wz0, leaf_heuristic<M>(x0, log2g, h_a0, h_b0, hz), h1);
          h1 = fmaf(wz1, leaf_heuristic<M>(x1, log2g, h_a0, h_b0, hz), h1);
          rs = fmaf(b.z, r0, rs);
          rs = fmaf(b.w, r1, rs);
        }
      }
      S0.add(s0);
      S1.add(s1);
      H.add(h1);
      R.add(rs);
    }
  }
  float s1, s0, h1;
  warp_sum4(S1.value(), S0.value(), H.value(), R.value(), s1, s0, h1, rbar_out);
  if (!(s1 >= kLinMinS1)) return false;
  lom_out = __logf((float)N) + kLn2 * (lg2(s1) - lg2(s0));
  v_out = h1 / s1;
  return true;
}

// The branch's sampled observation and representative come from the CTA's table (sm_ox,
// sm_oy, sm_rep), computed once per node.
template <class M>
__device__ void leaf_child_warp(const PlanDesc &P, const DevModel &dm, const SNode<M> &nb,
                                int l, unsigned long long node, int slot, float *sm_rb,
                                float *sm_lo, float *sm_v, const float *sm_ox,
                                const float *sm_oy, const int *sm_rep) {
  const int lane = threadIdx.x & 31, W = P.W;
  const int a = slot / W, k = slot - (slot / W) * W;
  const unsigned long long kn = key_node(P, l, node);
  const int j = sm_rep[slot];
  const typename M::O o = obs_from_f2<M>(make_float2(sm_ox[slot], sm_oy[slot]));
  const uint32_t c1 = key_level(P, l) | ((uint32_t)a << 8) | ((uint32_t)k << 16);
  float rbar, lom, v;
  if (P.branch_mode == kEnumerate || !leaf_sums_lin<M>(P, dm, nb, a, c1, kn, o, rbar, lom, v)) {
    if constexpr (kLogCold<M>::value) leaf_sums_log_cold<M>(P, dm, nb, a, c1, kn, o, rbar, lom, v);
    else leaf_sums_log<M>(P, dm, nb, a, c1, kn, o, rbar, lom, v);
  }
  if (lane == 0) {
    sm_rb[slot] = rbar;
    sm_lo[slot] = lom;
    sm_v[slot] = v;
    if (P.keep_leaf) {
      const unsigned long long c = node * (unsigned long long)P.AW + (unsigned long long)slot;
      P.rbar[l + 1][c] = rbar;
      P.lom[l + 1][c] = lom;
      P.V[l + 1][c] = v;
      if (P.keep_debug) {
        P.rep[l + 1][c] = j;
        const float2 of = M::obs_f2(o);
        P.obs[l + 1][2 * c] = of.x;
        P.obs[l + 1][2 * c + 1] = of.y;
      }
    }
  }
}

template <class M>
__device__ void leaf_item(const PlanDesc &P, unsigned long long node, float *smem, float *red,
                          bool fill_tables) {
  const DevModel &dm = *P.model;
  const int N = P.N, AW = P.AW, l = P.D - 1, npairs = (N + 1) >> 1;
  const SNode<M> nb = SNode<M>::at(smem, npairs);
  float *sm_rb = smem + (SNode<M>::kPairBytes / 4) * npairs;
  float *sm_lo = sm_rb + AW, *sm_v = sm_lo + AW;
  __shared__ float2 s_mu;
  if constexpr (std::is_same<M, GridModel>::value) {
    // the Z table and the tables by cell; x = 11 (exited) is the terminal column, its
    // heuristic 0 like a forced-zero one (a terminal state with x <= 10 exists only at the
    // root, with weight 0); the tables are read after the node build's barriers, and kept
    // from one work item to the next of the same plan
    if (fill_tables)
    for (int c = threadIdx.x; c < kGridCells; c += blockDim.x) {
      const int x = c & 15, y = c >> 4;
      const bool cell_ok = x <= 11 && y <= 10;
      for (int r = 0; r < 8; ++r) {
        const int dx = x - dm.rock_x[r], dy = y - dm.rock_y[r];
        const int d2 = cell_ok ? dx * dx + dy * dy : 0;
        s_grid_zc[r * kGridCells + c] = make_float2(dm.pz[d2], dm.pz[kGridD2 + d2]);
      }
      s_grid_rockc[c] = (signed char)((x <= 10 && y <= 10) ? dm.rock_at[x + 11 * y] : -1);
      const GridModel::S col{gpack(0, x <= 10 ? x : 0, 0, 0)};
      s_grid_hc[c] = (x <= 10 && P.h_zero == 0)
                         ? GridModel::heuristic(col, P.log2_gamma, P.h_a0, P.h_b0, false) : 0.0f;
    }
  }

  if (P.leaf_gen) {
    const unsigned long long parent = node / (unsigned long long)AW;
    const GNode<M> src = GNode<M>::at(P, l - 1, (long long)parent);
    float2 mu;
    typename M::O o;
    float lse2;
    build_child<M>(P, dm, l - 1, node, src, nb, ScratchInNode<M>{nb}, red, true, true, &mu, &o,
                   &lse2);
    if (threadIdx.x == 0) {
      s_mu = mu;
      if constexpr (std::is_same<M, GridModel>::value) {
        const int slot = (int)(node - parent * (unsigned long long)AW);
        s_grid_lw = GridLwCtx{src.lwp, nullptr, &dm, lse2, slot / P.W, o.o, N, 1};
      }
    }
  } else {
    const GNode<M> src = GNode<M>::at(P, l, (long long)node);
    if constexpr (std::is_same<M, GridModel>::value) {
      if (threadIdx.x == 0)
        s_grid_lw = GridLwCtx{nullptr, src.lwp, &dm, -CUDART_INF_F, 0, 0, N, 0};
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      nb.put(i, src.get(i));
      const float lw = src.lw(i);
      nb.set_lw(i, kLog2e * lw);                       // base 2 in shared memory
      nb.set_w(i, (lw > -CUDART_INF_F) ? __expf(lw) : 0.f);
      if constexpr (std::is_same<M, NavModel>::value)
        nb.set_m(i, NavModel::terminal(nb.get(i)) ? 0.0f : 1.0f);
    }
    if (threadIdx.x == 0)
      s_mu = (P.pi_mode == kPiNavDist) ? make_float2(P.mu[l][2 * node], P.mu[l][2 * node + 1])
                                       : make_float2(0.f, 0.f);
  }
  if ((N & 1) && threadIdx.x == 0) {   // odd N: the pad slot is a zero-weight copy of particle 0
    nb.put(N, nb.get(0));
    nb.set_lw(N, -CUDART_INF_F);
    nb.set_w(N, 0.f);
    if constexpr (std::is_same<M, NavModel>::value) nb.set_m(N, nb.m(0));
  }
  if (threadIdx.x < 10)   // the round keys of the plan's generator
    s_leaf_rk[threadIdx.x] = make_uint2(P.key0 + (uint32_t)threadIdx.x * 0x9E3779B9u,
                                        P.key1 + (uint32_t)threadIdx.x * 0xBB67AE85u);
  __syncthreads();

  // every branch's sampled observation and representative, one thread per branch (a
  // warp-uniform serial computation otherwise repeated by all 32 lanes of a branch's warp;
  // each warp drawing only its own branches' measured slower, 300 against 296 us)
  float *sm_ox = sm_v + AW, *sm_oy = sm_ox + AW;
  int *sm_rep = reinterpret_cast<int *>(sm_oy + AW);
  {
    const unsigned long long kn = key_node(P, l, node);
    for (int slot = threadIdx.x; slot < AW; slot += blockDim.x) {
      const int a = slot / P.W, k = slot - a * P.W;
      int j;
      const float2 of = M::obs_f2(branch_obs<M>(P, nb, l, a, k, kn, dm, j));
      sm_ox[slot] = of.x;
      sm_oy[slot] = of.y;
      sm_rep[slot] = j;
    }
  }
  __syncthreads();

  const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;

  for (int slot = wid; slot < AW; slot += nw)
    leaf_child_warp<M>(P, dm, nb, l, node, slot, sm_rb, sm_lo, sm_v, sm_ox, sm_oy, sm_rep);
  __syncthreads();

  if (wid == 0) {
    float q;
    // (at the root, depth 1, the preferences are updated once, by root_backup_warp)
    float *psi = (l > 0 && P.psi[l]) ? P.psi[l] + node * P.A : nullptr;
    const float v = node_backup_warp<false>(P, sm_rb, sm_lo, sm_v, s_mu, q, psi,
                                            l >= P.psi_new_level);
    const int lane = threadIdx.x & 31;
    if (lane < P.A) P.Q[l][node * P.A + lane] = q;
    if (lane == 0) P.V[l][node] = v;
    if (l == 0) {
      __threadfence_block();
      root_backup_warp(P);          // depth 1: this node is the root
    } else {
      climb_warp(P, l, node);
    }
  }
  __syncthreads();
}

// One leaf kernel per model, so that each gets its own register allocation and occupancy;
// a launch covers the leaf items of every plan of that model in one shared-memory class.
template <int K> struct LeafModel;
template <> struct LeafModel<kNav> { using type = NavModel; static constexpr int kMaxReg = VOPP_LEAF_NAV_MAXREG; };
template <> struct LeafModel<kGrid> { using type = GridModel; static constexpr int kMaxReg = VOPP_LEAF_GRID_MAXREG; };
template <> struct LeafModel<kToy> { using type = ToyModel; static constexpr int kMaxReg = VOPP_LEAF_TOY_MAXREG; };
template <> struct LeafModel<kCrowd> { using type = CrowdModel; };

template <int K>
__device__ __forceinline__ void leaf_kernel_body(const PlanDesc *plans, const StageTable &st,
                                                 long long total) {
  extern __shared__ __align__(16) float smem[];
  __shared__ float red[kRedFloats];
  __shared__ long long s_item;
  pdl_release_next();
  pdl_wait_prev();
  long long item = blockIdx.x;
  if (st.counter) {   // persistent CTAs: take work items in order from a global counter
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(st.counter, 1ull);
    __syncthreads();
    item = s_item;
    __syncthreads();
  }
  int tab_plan = -1;   // the plan whose model tables the CTA's shared memory holds
  while (item < total) {
    const int pi = find_plan(st, item);
    const PlanDesc &P = plans[st.plan[pi]];
    const unsigned long long node = (unsigned long long)(item - st.prefix[pi]);
    // persistent: the next item is taken now, its atomic's latency hidden by this item
    unsigned long long nxt = 0;
    if (st.counter && threadIdx.x == 0) nxt = atomicAdd(st.counter, 1ull);
    leaf_item<typename LeafModel<K>::type>(P, node, smem, red, pi != tab_plan);
    tab_plan = pi;
    if (st.counter) {
      if (threadIdx.x == 0) s_item = (long long)nxt;
      __syncthreads();
      item = s_item;
      __syncthreads();
    } else {
      item += gridDim.x;
    }
  }
}

// NAV2D, GRID, TOY2: a register cap per model; CROWD: its 160-thread CTAs, three per SM
template <int K>
__global__ void __maxnreg__(LeafModel<K>::kMaxReg)
k_leaf(const PlanDesc *plans, StageTable st, long long total) {
  leaf_kernel_body<K>(plans, st, total);
}
__global__ void __launch_bounds__(kCrowdLeafThreads, VOPP_LEAF_CROWD_MINBLOCKS)
k_leaf_crowd(const PlanDesc *plans, StageTable st, long long total) {
  leaf_kernel_body<kCrowd>(plans, st, total);
}

// ---------------------------------------------------------------------------------------
// K5: SIR belief update of one agent (one CTA, up to 65536 particles).
// ---------------------------------------------------------------------------------------
template <class M>
__device__ void belief_plan(const BeliefArgs &B, const DevModel &dm, float *red, double *dred) {
  const int N = B.N;
  GNode<M> cur, nxt;
  if constexpr (SelfDraw<M>::value) {
    cur = GNode<M>{B.x, B.y, B.pf, B.lw, B.s, N};
    nxt = GNode<M>{B.tx, B.ty, B.tpf, B.tlw, B.ts, N};
  } else if constexpr (M::kStochastic) {
    cur = GNode<M>{B.x, B.y, B.lw};
    nxt = GNode<M>{B.tx, B.ty, B.tlw};
  } else {
    cur.s = B.s; cur.lwp = B.lw;
    nxt.s = B.ts; nxt.lwp = B.tlw;
  }
  typename M::O o;
  if constexpr (M::kStochastic) o = typename M::O{B.obs_f[0], B.obs_f[1]};
  else o = typename M::O{B.obs_i};

  float m = -CUDART_INF_F;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    typename M::S s = cur.get(i);
    uint4 w = make_uint4(0u, 0u, 0u, 0u);
    if (M::kStochastic)
      w = draw(B.key0, B.key1, (uint32_t)(i >> 1), kPurposeBeliefStep, 0, 0, 0, B.t);
    step_particle<M>(s, B.action, w, i, DrawCtx{B.key0, B.key1, kPurposeBeliefStep, 0u, B.t}, dm);
    const float L = cur.lw(i) + M::loglik(s, B.action, o, dm);
    nxt.put(i, s);
    nxt.set_lw(i, L);
    m = fmaxf(m, L);
  }
  m = block_max(m, red);
  if (!(m > -CUDART_INF_F)) {
    if (threadIdx.x == 0) { B.out->status = 1; B.out->ess = 0.0; B.out->resampled = 0; }
    return;
  }
  Kahan S;
  S.init();
  for (int i = threadIdx.x; i < N; i += blockDim.x) S.add(__expf(nxt.lw(i) - m));
  const float lse = m + logf(block_sum(S.value(), red));
  Kahan Q2;
  Q2.init();
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const float nl = nxt.lw(i) - lse;
    nxt.set_lw(i, nl);
    const float w = __expf(nl);
    Q2.add(w * w);
  }
  const float sw2 = block_sum(Q2.value(), red);
  const float ess = 1.0f / sw2;
  const bool resample = ess < 0.5f * (float)N;

  if (resample) {
    // inclusive CDF in FP64: contiguous chunk per thread, then a block scan of chunk sums
    const int T = blockDim.x, tid = threadIdx.x;
    const int chunk = (N + T - 1) / T;
    const int b = tid * chunk, e = min(N, b + chunk);
    double acc = 0.0;
    for (int i = b; i < e; ++i) acc += (double)__expf(nxt.lw(i));
    dred[tid] = acc;
    __syncthreads();
    if (tid == 0) {
      double run = 0.0;
      for (int t = 0; t < T; ++t) { const double v = dred[t]; dred[t] = run; run += v; }
      dred[T] = run;
    }
    __syncthreads();
    double run = dred[tid];
    for (int i = b; i < e; ++i) { run += (double)__expf(nxt.lw(i)); B.cdf[i] = run; }
    __syncthreads();
    const double total = B.cdf[N - 1];
    const uint4 w = draw(B.key0, B.key1, 0u, kPurposeResample, 0, 0, 0, B.t);
    const double u0 = (double)u01(w.x);
    const float nlw = -logf((float)N);
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const double pos = (u0 + (double)i) / (double)N * total;
      int lo = 0, hi = N - 1;     // first k with pos < cdf[k], else N-1
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (pos < B.cdf[mid]) hi = mid; else lo = mid + 1;
      }
      B.anc[i] = lo;
      cur.put(i, nxt.get(lo));
      cur.set_lw(i, nlw);
    }
  } else {
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      cur.put(i, nxt.get(i));
      cur.set_lw(i, nxt.lw(i));
      B.anc[i] = i;
    }
  }
  if (threadIdx.x == 0) {
    B.out->status = 0;
    B.out->ess = (double)ess;
    B.out->resampled = resample ? 1 : 0;
  }
}

__global__ void __launch_bounds__(1024) k_belief(BeliefArgs B) {
  __shared__ float red[32];
  __shared__ double dred[1025];
  const DevModel &dm = *B.model;
  switch (B.kind) {
    case kNav: belief_plan<NavModel>(B, dm, red, dred); break;
    case kGrid: belief_plan<GridModel>(B, dm, red, dred); break;
    case kCrowd: belief_plan<CrowdModel>(B, dm, red, dred); break;
    default: belief_plan<ToyModel>(B, dm, red, dred); break;
  }
}

// Belief updates of many agents in one launch: CTA b updates agent b exactly as k_belief
// would (same block size, same reduction order).
__global__ void __launch_bounds__(1024) k_belief_batch(const BeliefArgs *args) {
  __shared__ float red[32];
  __shared__ double dred[1025];
  const BeliefArgs &B = args[blockIdx.x];
  const DevModel &dm = *B.model;
  switch (B.kind) {
    case kNav: belief_plan<NavModel>(B, dm, red, dred); break;
    case kGrid: belief_plan<GridModel>(B, dm, red, dred); break;
    case kCrowd: belief_plan<CrowdModel>(B, dm, red, dred); break;
    default: belief_plan<ToyModel>(B, dm, red, dred); break;
  }
}

// ---------------------------------------------------------------------------------------
// K7: one environment step of the closed loop (Alg. 1: execute the action, perceive the
// observation).  The true state steps under the model's own transition and observation
// processes with random numbers of its own: Philox purpose 5 (transition words 0,1) and 6
// (observation words 0,1), node word = the environment's time step.
// ---------------------------------------------------------------------------------------
template <class M>
__device__ void env_step(const EnvArgs &E) {
  const DevModel &dm = *E.model;
  typename M::S s;
  if constexpr (SelfDraw<M>::value) {
    s.x = E.xy[0];
    s.y = E.xy[1];
    for (int q = 0; q < 12; ++q) (q & 1 ? s.py : s.px)[q >> 1] = E.pf[q];
    s.f = E.s[0];
  } else if constexpr (M::kStochastic) {
    s = typename M::S{E.xy[0], E.xy[1]};
  } else {
    s = typename M::S{E.s[0]};
  }
  const uint4 w = draw(E.key0, E.key1, 0u, kPurposeEnvStep, 0, 0, 0, E.t);
  const float r = step_particle<M>(s, E.action, w, 0, DrawCtx{E.key0, E.key1, kPurposeEnvStep, 0u, E.t}, dm);
  const uint4 v = draw(E.key0, E.key1, 0u, kPurposeEnvObs, 0, 0, 0, E.t);
  const typename M::O o =
      obs_particle<M>(s, E.action, v, DrawCtx{E.key0, E.key1, kPurposeEnvObs, 0u, E.t}, 0u, dm);
  if constexpr (SelfDraw<M>::value) {
    E.xy[0] = s.x;
    E.xy[1] = s.y;
    for (int q = 0; q < 12; ++q) E.pf[q] = (q & 1 ? s.py : s.px)[q >> 1];
    E.s[0] = s.f;
    E.out->obs[0] = (float)o.o;
    E.out->obs[1] = 0.f;
    E.out->obs_i = o.o;
  } else if constexpr (M::kStochastic) {
    E.xy[0] = s.x;
    E.xy[1] = s.y;
    E.out->obs[0] = o.x;
    E.out->obs[1] = o.y;
    E.out->obs_i = 0;
  } else {
    E.s[0] = s.s;
    E.out->obs[0] = (float)o.o;
    E.out->obs[1] = 0.f;
    E.out->obs_i = o.o;
  }
  E.out->reward = r;
  E.out->terminal = M::terminal(s) ? 1 : 0;
}

__global__ void k_env(EnvArgs E) {
  if (threadIdx.x != 0) return;
  switch (E.kind) {
    case kNav: env_step<NavModel>(E); break;
    case kGrid: env_step<GridModel>(E); break;
    case kCrowd: env_step<CrowdModel>(E); break;
    default: env_step<ToyModel>(E); break;
  }
}

// ---------------------------------------------------------------------------------------
// Host-side launchers.
// ---------------------------------------------------------------------------------------
size_t leaf_smem_bytes(int kind, int N, int AW) {
  const size_t pair = (kind == kNav) ? SNode<NavModel>::kPairBytes
                                     : kind == kCrowd ? SNode<CrowdModel>::kPairBytes
                                     : kind == kGrid ? SNode<GridModel>::kPairBytes : 24;
  // node pairs; per branch: r̄, log ω, V, and the sampled observation (2 floats) with its
  // representative
  return pair * (size_t)((N + 1) / 2) + 6 * sizeof(float) * (size_t)AW + 64;
}
size_t expand_smem_bytes(int N) { return 8 * (size_t)N + 64; }
size_t root_node_words(int kind) { return kind == kNav ? 3 : (kind == kCrowd ? 16 : 2); }
size_t expand_fused_smem_bytes(int kind, int N) {
  return expand_smem_bytes(N) + 4 * root_node_words(kind) * (size_t)N;
}

cudaError_t launch_root_prep(const PlanDesc *d, const StageTable &st, cudaStream_t s) {
  k_root_prep<<<st.n_plans, 1024, 0, s>>>(d, st);
  return cudaGetLastError();
}

// Dynamic shared memory ceilings of the kernels that may exceed 48 KB (set once, before any
// stream capture).
cudaError_t init_kernel_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_expand<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kLeafSmemLimit);
  if (e == cudaSuccess && kExpandWide > 256)
    e = cudaFuncSetAttribute(k_expand<kExpandWide>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kLeafSmemLimit);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_leaf<kNav>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kLeafSmemLimit);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_leaf<kGrid>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kLeafSmemLimit);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_leaf<kToy>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kLeafSmemLimit);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_leaf_crowd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kLeafSmemLimit);
  return e;
}

// Launch with programmatic stream serialisation: the kernel may be scheduled while its
// predecessor on the stream is still running and waits for it on the device.
template <typename... Args>
static cudaError_t launch_pdl(void (*k)(Args...), unsigned grid, unsigned threads, size_t smem,
                              cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

cudaError_t launch_expand(const PlanDesc *d, const StageTable &st, long long total, size_t smem,
                          long long grid, bool wide, cudaStream_t s) {
  if (kExpandWide > 256 && wide)
    return launch_pdl(k_expand<kExpandWide>, (unsigned)grid, (unsigned)kExpandWide, smem, s, d, st, total);
  return launch_pdl(k_expand<256>, (unsigned)grid, 256u, smem, s, d, st, total);
}

cudaError_t launch_expand_vec(int kind, int vw, const PlanDesc *d, const StageTable &st,
                              long long total, long long grid, cudaStream_t s) {
  static_assert(kExpandVecWarps == kExpandVecChildrenPerCta, "one child per warp");
  const unsigned g = (unsigned)grid, t = (unsigned)kExpandVecThreads;
#define VOPP_EXPAND_VEC_CASE(K)                                                      \
  if (kind == K) {                                                                   \
    if (vw == 4) return launch_pdl(k_expand_vec<K, 4>, g, t, 0, s, d, st, total);    \
    if (vw == 2) return launch_pdl(k_expand_vec<K, 2>, g, t, 0, s, d, st, total);    \
    return launch_pdl(k_expand_vec<K, 1>, g, t, 0, s, d, st, total);                 \
  }
  VOPP_EXPAND_VEC_CASE(kNav)
  VOPP_EXPAND_VEC_CASE(kGrid)
  VOPP_EXPAND_VEC_CASE(kToy)
#undef VOPP_EXPAND_VEC_CASE
  return cudaErrorInvalidValue;
}



cudaError_t launch_leaf(int kind, const PlanDesc *d, const StageTable &st, long long total,
                        size_t smem, int threads, long long grid, cudaStream_t s) {
  switch (kind) {
    case kNav: return launch_pdl(k_leaf<kNav>, (unsigned)grid, (unsigned)threads, smem, s, d, st, total);
    case kGrid: return launch_pdl(k_leaf<kGrid>, (unsigned)grid, (unsigned)threads, smem, s, d, st, total);
    case kToy: return launch_pdl(k_leaf<kToy>, (unsigned)grid, (unsigned)threads, smem, s, d, st, total);
    case kCrowd: return launch_pdl(k_leaf_crowd, (unsigned)grid, (unsigned)kCrowdLeafThreads, smem, s, d, st, total);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t leaf_occupancy(int kind, int threads, size_t smem, int *blocks_per_sm) {
  switch (kind) {
    case kNav: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_leaf<kNav>, threads, smem);
    case kGrid: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_leaf<kGrid>, threads, smem);
    case kToy: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_leaf<kToy>, threads, smem);
    case kCrowd: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_leaf_crowd, kCrowdLeafThreads, smem);
    default: return cudaErrorInvalidValue;
  }
}

// Copy i of the list in slices of kCopySlice bytes, one CTA per (copy, slice): 16-byte words
// where both ends and the size allow, else 4-byte words.
// Slice blockIdx.y (and every gridDim.y-th after it) of one copy, by one CTA.
__device__ __forceinline__ void copy_slices(void *dst, const void *src, unsigned long long bytes) {
  char *d = static_cast<char *>(dst);
  const char *sp = static_cast<const char *>(src);
  const bool v16 = ((reinterpret_cast<uintptr_t>(d) | reinterpret_cast<uintptr_t>(sp) | bytes) & 15) == 0;
  for (unsigned long long lo = (unsigned long long)blockIdx.y * kCopySlice; lo < bytes;
       lo += (unsigned long long)gridDim.y * kCopySlice) {
    const unsigned long long hi = min(bytes, lo + kCopySlice);
    if (v16) {
      uint4 *d4 = reinterpret_cast<uint4 *>(d);
      const uint4 *s4 = reinterpret_cast<const uint4 *>(sp);
      for (unsigned long long w = lo / 16 + threadIdx.x; w < hi / 16; w += blockDim.x)
        d4[w] = sp ? s4[w] : make_uint4(0u, 0u, 0u, 0u);
    } else {
      uint32_t *d1 = reinterpret_cast<uint32_t *>(d);
      const uint32_t *s1 = reinterpret_cast<const uint32_t *>(sp);
      for (unsigned long long w = lo / 4 + threadIdx.x; w < hi / 4; w += blockDim.x) d1[w] = sp ? s1[w] : 0u;
    }
  }
}
__global__ void __launch_bounds__(256) k_copy_list(CopyList L) {
  const int i = blockIdx.x;
  if (i < L.n) copy_slices(L.dst[i], L.src[i], L.bytes[i]);
}
__global__ void __launch_bounds__(256) k_copy_table(const CopyDesc *t, int n) {
  const int i = blockIdx.x;
  if (i < n) copy_slices(t[i].dst, t[i].src, t[i].bytes);
}

// Root preparation and the copies of continued subtrees in one launch (see the declaration).
// The copies of levels >= 1 read only the kept stores and write only levels the root
// preparation does not touch, so the two kinds of CTA need no order between them.
__global__ void __launch_bounds__(1024) k_root_prep_copy(const PlanDesc *plans, StageTable st,
                                                         const CopyDesc *t, int n_rest,
                                                         unsigned slices) {
  __shared__ float red[128];
  pdl_release_next();
  const unsigned b = blockIdx.x;
  if (b >= (unsigned)st.n_plans) {   // a slice of one of the other copies
    copy_table_slice(t, n_rest, slices, b - (unsigned)st.n_plans);
    return;
  }
  const PlanDesc &P = plans[st.plan[b]];
  if (P.copy0_n > 0) {   // the root's particles and log weights, before the root reads them
    for (int q = P.copy0_first; q < P.copy0_first + P.copy0_n; ++q) copy_cta(t[q].dst, t[q].src, t[q].bytes);
    __syncthreads();
  }
  const DevModel &dm = *P.model;
  switch (P.kind) {
    case kNav: root_prep_plan<NavModel>(P, dm, red); break;
    case kGrid: root_prep_plan<GridModel>(P, dm, red); break;
    case kCrowd: root_prep_plan<CrowdModel>(P, dm, red); break;
    default: root_prep_plan<ToyModel>(P, dm, red); break;
  }
}

static unsigned copy_slice_count(unsigned long long most) {
  return (unsigned)std::min<unsigned long long>(
      65535, std::max<unsigned long long>(1, (most + kCopySlice - 1) / kCopySlice));
}

cudaError_t launch_copy_table(const CopyDesc *table, int n, unsigned long long most, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_copy_table<<<dim3((unsigned)n, copy_slice_count(most)), 256, 0, s>>>(table, n);
  return cudaGetLastError();
}

cudaError_t launch_root_prep_copy(const PlanDesc *d, const StageTable &st, const CopyDesc *table,
                                  int n_rest, unsigned long long most, cudaStream_t s) {
  // 64 KB slices of every other copy: at most 65,535 of them per copy (as the copy table)
  const unsigned slices = n_rest > 0 ? (unsigned)std::min<unsigned long long>(
                                           65535, std::max<unsigned long long>(1, (most + kCopySlice - 1) / kCopySlice))
                                     : 1u;
  const unsigned long long grid = (unsigned long long)st.n_plans + (unsigned long long)n_rest * slices;
  if (grid == 0 || grid > 0x7fffffffull) return cudaErrorInvalidValue;
  k_root_prep_copy<<<(unsigned)grid, 1024, 0, s>>>(d, st, table, n_rest, slices);
  return cudaGetLastError();
}

cudaError_t launch_copy_list(const CopyList &L, cudaStream_t s) {
  if (L.n <= 0) return cudaSuccess;
  unsigned long long most = 0;
  for (int i = 0; i < L.n; ++i) most = std::max(most, L.bytes[i]);
  k_copy_list<<<dim3((unsigned)L.n, copy_slice_count(most)), 256, 0, s>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_env(const EnvArgs &E, cudaStream_t s) {
  k_env<<<1, 32, 0, s>>>(E);
  return cudaGetLastError();
}

cudaError_t launch_belief(const BeliefArgs &B, cudaStream_t s) {
  k_belief<<<1, 1024, 0, s>>>(B);
  return cudaGetLastError();
}

cudaError_t launch_belief_batch(const BeliefArgs *d_args, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_belief_batch<<<n, 1024, 0, s>>>(d_args);
  return cudaGetLastError();
}

}  // namespace vopp
